"""FP64 CPU oracle: two-component (spinor) PSTD run with a sigma . B coupling.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper motivates the method with magnetic (spin-dependent) scattering but works with a
scalar wave function; this is the spinor generalisation of the oracle's leapfrog, step by step
as in pstd_oracle.Simulation, with the Hamiltonian
    H = -hbar^2/2m lap + V(r) I + gamma sigma . B(r),
    sigma . B = [[Bz, Bx - i By], [Bx + i By, -Bz]],
in the EXACT TF/SF form: the state u = (u_up, u_down) is the scattered spinor and the incident
spinor chi psi_inc (chi = incident spin state, psi_inc the scalar plane wave of Simulation) enters
through W (u + chi psi_inc), W = V I + gamma sigma . B.  Each component's phasors are scaled by
the incident phasor of the scalar wave at r_O (so spin-flip amplitudes are defined when chi has a
zero component).
"""
from __future__ import annotations

import math

import numpy as np

from .pstd_oracle import (AXES_NP, Simulation, apply_axis, coords, envelope, eta, first_contact_corner, kinetic,
                          mask_1d)


def coupling(V, B, gamma):
    """W = V I + gamma sigma . B as its four [z, y, x] blocks (W_uu, W_ud, W_du, W_dd)."""
    Bx, By, Bz = (np.asarray(b, dtype=np.float64) for b in B)
    return (V + gamma * Bz, gamma * (Bx - 1j * By), gamma * (Bx + 1j * By), V - gamma * Bz)


class SpinorSimulation:
    """Leapfrog PSTD of a two-component wave function (EXACT TF/SF form)."""

    def __init__(self, spec, V, B, gamma, khat, k, ramp_time, chi, window=None, omegas=None):
        if spec.tfsf_mode != "exact":
            raise ValueError("the spinor oracle uses the EXACT TF/SF form")
        # the scalar machinery (tables, incident wave, DFT) of each component, with V = 0: the
        # interaction is applied here
        self.comp = [Simulation(spec, np.zeros(spec.shape), khat, k, ramp_time, window=window, omegas=omegas)
                     for _ in range(2)]
        self.spec = spec
        self.W = coupling(V, B, gamma)
        self.chi = (complex(chi[0]), complex(chi[1]))
        self.n = 0

    def _advance(self):
        s0, s1 = self.comp
        spec = s0.spec
        c = 2j * spec.dt / spec.hbar
        pinc = s0.psi_inc(self.n)
        tot = [s0.cur + self.chi[0] * pinc, s1.cur + self.chi[1] * pinc]
        Wuu, Wud, Wdu, Wdd = self.W
        Hu = [s0.kin_coef * kinetic(s0.cur, spec.d) + Wuu * tot[0] + Wud * tot[1],
              s1.kin_coef * kinetic(s1.cur, spec.d) + Wdu * tot[0] + Wdd * tot[1]]
        return [s.Gamma * (s.prev - c * h) for s, h in zip(self.comp, Hu)]

    def step(self, count: int = 1):
        for _ in range(count):
            for s in self.comp:
                if s.in_window(s.n):
                    s.accumulate()
            nxt = self._advance()
            for s, v in zip(self.comp, nxt):
                s.prev, s.cur = s.cur, v
                s.n += 1
            self.n += 1

    @property
    def cur(self):
        return [s.cur for s in self.comp]

    def scaled_phasors(self, component: int, fi: int = 0):
        """Phasors of one component over the scalar incident phasor at r_O."""
        return self.comp[component].scaled_phasors(fi)


def eigen_spin(nhat):
    """Eigenvectors of sigma . nhat for a unit vector nhat: (+1 eigenvector, -1 eigenvector)."""
    nx, ny, nz = nhat
    M = np.array([[nz, nx - 1j * ny], [nx + 1j * ny, -nz]])
    w, v = np.linalg.eigh(M)
    return v[:, 1], v[:, 0]


def kinetic_at(u, d, node):
    """(K u) at one node (i, j, k) of a [z, y, x] array from the three grid lines through it: the
    spectral Laplacian of Eq. spatialFFTeigen is a sum of one-axis operators, so each term needs
    only the line along its axis."""
    i, j, k = node
    lines = (u[k, j, :], u[k, :, i], u[:, j, i])
    out = 0j
    for a in range(3):
        shp = [1, 1, 1]
        shp[AXES_NP[a]] = -1
        line = np.asarray(lines[a], dtype=np.complex128).reshape(shp)
        pos = (i, j, k)[a]
        out += complex(apply_axis(line, a, d[a], lambda q: q * q).ravel()[pos])
    return out


def step_at_nodes(spec, V, B, gamma, khat, k, ramp_time, chi, prev, cur, n, nodes):
    """psi^{n+1} of both spinor components at the given nodes (i, j, k), the update of
    SpinorSimulation evaluated node by node (for grids too large for the whole-array oracle).

    prev, cur: pairs of [z, y, x] arrays (up, down) at levels n-1 and n; V, B: the potential and
    the three induction components, [z, y, x] arrays.  Returns a (len(nodes), 2) complex array."""
    hb, m = spec.hbar, spec.mass
    kh = np.asarray(khat, dtype=float) / np.linalg.norm(khat)
    E0 = hb * hb * k * k / (2.0 * m)
    w0 = E0 / hb
    kin_coef = hb * hb / (2.0 * m) * eta(E0, spec.dt, hb)
    gam = [mask_1d(spec.n[a], spec.abc_cells[a], spec.abc_profile, spec.abc_param, E0, spec.dt, hb) for a in range(3)]
    rO = first_contact_corner(kh, spec)
    x = [coords(spec.n[a], spec.d[a]) for a in range(3)]
    t = n * spec.dt
    tf = envelope(t, ramp_time) * complex(math.cos(w0 * t), -math.sin(w0 * t))
    c = 2j * spec.dt / hb
    ch = (complex(chi[0]), complex(chi[1]))
    out = np.zeros((len(nodes), 2), dtype=np.complex128)
    for q, (i, j, kk) in enumerate(nodes):
        r = np.array([x[0][i], x[1][j], x[2][kk]])
        pinc = tf * complex(np.exp(1j * k * float(kh @ (r - rO))))
        Wuu, Wud, Wdu, Wdd = coupling(V[kk, j, i], [b[kk, j, i] for b in B], gamma)
        tot = [complex(cur[0][kk, j, i]) + ch[0] * pinc, complex(cur[1][kk, j, i]) + ch[1] * pinc]
        H = [kin_coef * kinetic_at(cur[0], spec.d, (i, j, kk)) + Wuu * tot[0] + Wud * tot[1],
             kin_coef * kinetic_at(cur[1], spec.d, (i, j, kk)) + Wdu * tot[0] + Wdd * tot[1]]
        G = gam[0][i] * gam[1][j] * gam[2][kk]
        for s in range(2):
            out[q, s] = G * (complex(prev[s][kk, j, i]) - c * H[s])
    return out

