"""Closed forms that pin the oracle to something other than itself.

TEST INFRASTRUCTURE ONLY (see the package docstring).

  * partial-wave scattering amplitude of a central square potential (the paper's
    golden standard, Section 4, Eq. sphericalV; textbook phase shifts)
  * first Born amplitude of a voxel potential (the usual approximate method the
    paper names in its introduction)
  * outgoing spherical wave e^{ik|r - r_s|}/|r - r_s| and its gradient (the NTDF
    validation field of Section 3.4)
  * leapfrog evolution of one Fourier mode (Eqs. tempeigen, q_equation, Joukowsky)
"""
from __future__ import annotations

import math

import numpy as np
from scipy import special


def phase_shifts(k: float, V0: float, a: float, hbar: float = 1.0, mass: float = 1.0, lmax: int | None = None):
    """delta_l for V = V0 (r <= a), 0 outside, matching log-derivatives at r = a.

    tan delta_l = [k j_l'(ka) - g_l j_l(ka)] / [k y_l'(ka) - g_l y_l(ka)], with g_l the
    interior log-derivative: K j_l'(Ka)/j_l(Ka) (E > V0), kappa i_l'(kappa a)/i_l(kappa a)
    (E < V0), l/a (E = V0).
    """
    E = hbar * hbar * k * k / (2.0 * mass)
    if lmax is None:
        lmax = int(k * a + 25)
    K2 = 2.0 * mass * (E - V0) / (hbar * hbar)
    ls = np.arange(lmax + 1)
    ka = k * a
    if K2 > 0:
        K = math.sqrt(K2)
        g = K * special.spherical_jn(ls, K * a, derivative=True) / special.spherical_jn(ls, K * a)
    elif K2 < 0:
        kap = math.sqrt(-K2)
        g = kap * special.spherical_in(ls, kap * a, derivative=True) / special.spherical_in(ls, kap * a)
    else:
        g = ls / a
    num = k * special.spherical_jn(ls, ka, derivative=True) - g * special.spherical_jn(ls, ka)
    den = k * special.spherical_yn(ls, ka, derivative=True) - g * special.spherical_yn(ls, ka)
    # delta_l is fixed modulo pi, which leaves e^{i delta} sin(delta) unchanged
    return np.arctan(num / den)


def partial_wave_amplitude(theta, k: float, V0: float, a: float, hbar: float = 1.0, mass: float = 1.0,
                           lmax: int | None = None) -> np.ndarray:
    """f(theta) = (1/k) sum_l (2l+1) e^{i delta_l} sin(delta_l) P_l(cos theta) (incident e^{ikz})."""
    d = phase_shifts(k, V0, a, hbar, mass, lmax)
    ls = np.arange(len(d))
    x = np.cos(np.atleast_1d(theta))
    P = special.eval_legendre(ls[:, None], x[None, :])
    coef = (2 * ls + 1) * np.exp(1j * d) * np.sin(d) / k
    return coef @ P


def born_amplitude(V: np.ndarray, xyz_axes, dV: float, k_in, k_out, hbar: float = 1.0, mass: float = 1.0):
    """f_B = -(m / 2 pi hbar^2) sum_nodes V e^{-i q . r} dV, q = k_out - k_in (incident e^{i k_in . r})."""
    x, y, z = xyz_axes
    k_in = np.asarray(k_in, dtype=float)
    out = []
    for ko in np.atleast_2d(k_out):
        q = ko - k_in
        ex = np.exp(-1j * q[0] * x)
        ey = np.exp(-1j * q[1] * y)
        ez = np.exp(-1j * q[2] * z)
        s = np.einsum("kji,k,j,i->", V, ez, ey, ex)
        out.append(-mass / (2 * math.pi * hbar * hbar) * s * dV)
    return np.array(out)


def spherical_wave(points, k: float, src=(0.0, 0.0, 0.0)):
    """psi = e^{ik rho}/rho and grad psi = (ik - 1/rho) e^{ik rho}/rho * (r - src)/rho."""
    p = np.atleast_2d(np.asarray(points, dtype=float)) - np.asarray(src, dtype=float)
    rho = np.linalg.norm(p, axis=1)
    psi = np.exp(1j * k * rho) / rho
    grad = ((1j * k - 1.0 / rho) * psi / rho)[:, None] * p
    return psi, grad


def leapfrog_mode_frequency(kk2: float, dt: float, eta: float, hbar: float = 1.0, mass: float = 1.0,
                            V: float = 0.0) -> float:
    """Discrete angular frequency of a Fourier mode with |k|^2 = kk2 under the leapfrog.

    psi^{n+1} - psi^{n-1} = -(2 i dt / hbar) lambda psi^n with lambda = eta hbar^2 kk2 / 2m + V and
    psi^n = e^{-i w n dt} gives sin(w dt) = lambda dt / hbar (Eq. q_equation with |q| = 1).
    """
    lam = eta * hbar * hbar * kk2 / (2.0 * mass) + V
    return math.asin(lam * dt / hbar) / dt


def leapfrog_growth(kk2: float, dt: float, eta: float, hbar: float = 1.0, mass: float = 1.0, V: float = 0.0) -> float:
    """|q| of the growing root when w = lambda dt / hbar exceeds 1: |Q| = w + sqrt(w^2 - 1) (Eq. Joukowsky)."""
    w = (eta * hbar * hbar * kk2 / (2.0 * mass) + V) * dt / hbar
    return w + math.sqrt(max(w * w - 1.0, 0.0))


def radial_phase_shifts(k: float, Vfun, r_max: float, hbar: float = 1.0, mass: float = 1.0,
                        lmax: int | None = None, rtol: float = 1e-11):
    """delta_l of a smooth central potential V(r) (V ~ 0 beyond r_max) by integrating the
    radial equation u'' = [l(l+1)/r^2 + 2m V(r)/hbar^2 - k^2] u outward and matching the
    log-derivative to j_l, y_l at r_max (the partial-wave method the paper takes as its
    golden standard, Section 4)."""
    from scipy.integrate import solve_ivp
    if lmax is None:
        lmax = int(k * r_max + 25)
    out = np.zeros(lmax + 1)
    for l in range(lmax + 1):
        r0 = min(1e-3 * (l + 1), 0.5 * r_max)

        def rhs(r, y):
            u, du = y
            return [du, (l * (l + 1) / (r * r) + 2.0 * mass * Vfun(r) / (hbar * hbar) - k * k) * u]

        sol = solve_ivp(rhs, (r0, r_max), [1.0, (l + 1) / r0], method="DOP853", rtol=rtol, atol=1e-300)
        u, du = sol.y[0, -1], sol.y[1, -1]
        g = du / u - 1.0 / r_max        # R'/R with R = u / r
        x = k * r_max
        num = k * special.spherical_jn(l, x, derivative=True) - g * special.spherical_jn(l, x)
        den = k * special.spherical_yn(l, x, derivative=True) - g * special.spherical_yn(l, x)
        out[l] = np.arctan(num / den)
    return out


def amplitude_from_phase_shifts(theta, k: float, delta) -> np.ndarray:
    ls = np.arange(len(delta))
    x = np.cos(np.atleast_1d(theta))
    P = special.eval_legendre(ls[:, None], x[None, :])
    return ((2 * ls + 1) * np.exp(1j * delta) * np.sin(delta) / k) @ P
