"""FP64 CPU oracle: near-to-distant-field transform (Section 3).

TEST INFRASTRUCTURE ONLY (see the package docstring).

The transform is the literal per-cell mode sum of Eqs. bottomPsi_lm, topPsi_lm,
backfrontPsi_mn, leftrightPsi_ln summed over the six faces (Eq. Psi):

  Psi_cell(r) = -sigma * (D_b D_c e^{ikR}) / (4 pi N_b N_c R)
                * sum_{i',j'} (-1)^{i'+j'} e^{2 pi i (i' x^c / L_b + j' y^c / L_c)}
                  { F[d psi/d a]_{i'j'} + (ik - 1/R) (Rhat . a) F[psi]_{i'j'} }
                  sinc(pi i'/N_b - k D_b Rhat_b / 2) sinc(pi j'/N_c - k D_c Rhat_c / 2)

with sigma = -1 on the face at the low end of the normal axis a (bottom, back,
left: the "+" sign in the paper) and +1 at the high end (top, front, right),
sinc(x) = sin(x)/x, the 2-D FFT F taken over the whole virtual plane
(Eq. AnBottomPsi), and the cells (l, m) those between the nodes of the virtual
surface.  The far-field amplitude is the r -> infinity limit of the same sum,
f(rhat) = lim r e^{-ikr} Psi(r rhat): e^{ikR}/R -> e^{-ik rhat . r_c}, Rhat -> rhat,
(ik - 1/R) -> ik (the far-field form of Eq. FDTDfarfieldapprox applied per cell).
"""
from __future__ import annotations

import math

import numpy as np

from .pstd_oracle import FACES, coords, in_plane_axes


def _usinc(x):
    """Unnormalised sinc(x) = sin(x)/x."""
    return np.sinc(np.asarray(x) / math.pi)


def _face_setup(spec, face: int):
    a, s = FACES[face]
    b, c = in_plane_axes(a)
    h = spec.huygens_lo[a] if s == 0 else spec.huygens_hi[a]
    plane_coord = coords(spec.n[a], spec.d[a])[h]
    sigma = -1.0 if s == 0 else 1.0
    Nb, Nc = spec.n[b], spec.n[c]
    Db, Dc = spec.d[b], spec.d[c]
    xb = coords(Nb, Db)
    xc = coords(Nc, Dc)
    lb = np.arange(spec.huygens_lo[b], spec.huygens_hi[b])
    lc = np.arange(spec.huygens_lo[c], spec.huygens_hi[c])
    cb = xb[lb] + 0.5 * Db            # cell centres x^c_l = (x_l + x_{l+1}) / 2
    cc = xc[lc] + 0.5 * Dc
    ib = np.rint(np.fft.fftfreq(Nb) * Nb)   # i' in -N/2..N/2-1 (FFT order)
    ic = np.rint(np.fft.fftfreq(Nc) * Nc)
    sgn_b = 1.0 - 2.0 * np.mod(ib, 2)       # (-1)^{i'}
    sgn_c = 1.0 - 2.0 * np.mod(ic, 2)
    eb = sgn_b[None, :] * np.exp(2j * math.pi * ib[None, :] * cb[:, None] / (Nb * Db))   # [l, i']
    ec = sgn_c[None, :] * np.exp(2j * math.pi * ic[None, :] * cc[:, None] / (Nc * Dc))   # [m, j']
    return dict(a=a, b=b, c=c, sigma=sigma, plane_coord=plane_coord, Nb=Nb, Nc=Nc, Db=Db, Dc=Dc,
                cb=cb, cc=cc, ib=ib, ic=ic, eb=eb, ec=ec)


def transform_to_points(spec, k: float, phasors, points) -> np.ndarray:
    """Psi(r) at each row of `points` (M x 3) from the six scaled plane phasor pairs.

    phasors: list of 6 (psi_plane, dpsi_plane), planes as returned by
    pstd_oracle.plane_slice (array [slow, fast] = [c, b]); dpsi is the derivative along
    the plane's normal axis a (not along the outward normal).
    """
    pts = np.atleast_2d(np.asarray(points, dtype=float))
    out = np.zeros(len(pts), dtype=np.complex128)
    for face in range(6):
        g = _face_setup(spec, face)
        psi, dpsi = phasors[face]
        Cp = np.fft.fft2(psi)     # [j', i']
        Cd = np.fft.fft2(dpsi)
        a, b, c = g["a"], g["b"], g["c"]
        L, M = len(g["cb"]), len(g["cc"])
        pref = -g["sigma"] * g["Db"] * g["Dc"] / (4.0 * math.pi * g["Nb"] * g["Nc"])
        for p, r in enumerate(pts):
            Rb = r[b] - g["cb"][:, None] + 0.0 * g["cc"][None, :]     # [l, m]
            Rc = r[c] - g["cc"][None, :] + 0.0 * g["cb"][:, None]
            Ra = np.full((L, M), r[a] - g["plane_coord"])
            R = np.sqrt(Ra * Ra + Rb * Rb + Rc * Rc)
            hb_, hc_, ha_ = Rb / R, Rc / R, Ra / R
            sb = _usinc(math.pi * g["ib"][None, None, :] / g["Nb"] - 0.5 * k * g["Db"] * hb_[:, :, None])  # [l,m,i']
            sc = _usinc(math.pi * g["ic"][None, None, :] / g["Nc"] - 0.5 * k * g["Dc"] * hc_[:, :, None])  # [l,m,j']
            A = (g["eb"][:, None, :] * sb).reshape(L * M, g["Nb"])
            B = (g["ec"][None, :, :] * sc).reshape(L * M, g["Nc"])
            Sp = np.sum((A @ Cp.T) * B, axis=1).reshape(L, M)
            Sd = np.sum((A @ Cd.T) * B, axis=1).reshape(L, M)
            term = pref * np.exp(1j * k * R) / R * (Sd + (1j * k - 1.0 / R) * ha_ * Sp)
            out[p] += term.sum()
    return out


def far_field_amplitude(spec, k: float, phasors, theta, phi) -> np.ndarray:
    """f(theta, phi) = lim r e^{-ikr} Psi(r rhat); dsigma/dOmega = |f|^2."""
    th = np.atleast_1d(np.asarray(theta, dtype=float))
    ph = np.atleast_1d(np.asarray(phi, dtype=float))
    rh = np.stack([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)], axis=1)
    out = np.zeros(len(rh), dtype=np.complex128)
    for face in range(6):
        g = _face_setup(spec, face)
        psi, dpsi = phasors[face]
        Cp = np.fft.fft2(psi)
        Cd = np.fft.fft2(dpsi)
        a, b, c = g["a"], g["b"], g["c"]
        pref = -g["sigma"] * g["Db"] * g["Dc"] / (4.0 * math.pi * g["Nb"] * g["Nc"])
        for p, u in enumerate(rh):
            sb = _usinc(math.pi * g["ib"] / g["Nb"] - 0.5 * k * g["Db"] * u[b])     # [i']
            sc = _usinc(math.pi * g["ic"] / g["Nc"] - 0.5 * k * g["Dc"] * u[c])     # [j']
            A = g["eb"] * sb[None, :]        # [l, i']
            B = g["ec"] * sc[None, :]        # [m, j']
            Sp = (A @ Cp.T) @ B.T            # [l, m]
            Sd = (A @ Cd.T) @ B.T
            phase = np.exp(-1j * k * (u[a] * g["plane_coord"] + u[b] * g["cb"][:, None] + u[c] * g["cc"][None, :]))
            out[p] += (pref * phase * (Sd + 1j * k * u[a] * Sp)).sum()
    return out


def cross_section(spec, k, phasors, theta, phi):
    f = far_field_amplitude(spec, k, phasors, theta, phi)
    return np.abs(f) ** 2, f


def interpolant(plane: np.ndarray, Nb: int, Nc: int, Db: float, Dc: float, xb, xc) -> np.ndarray:
    """psi_an at (xb[p], xc[p]) from its definition (Eq. AnBottomPsi), by the direct double sum."""
    C = np.fft.fft2(plane)
    ib = np.rint(np.fft.fftfreq(Nb) * Nb)
    ic = np.rint(np.fft.fftfreq(Nc) * Nc)
    Lb, Lc = Nb * Db, Nc * Dc
    eb = np.exp(2j * math.pi * ib[None, :] * (np.asarray(xb)[:, None] + Lb / 2) / Lb)
    ec = np.exp(2j * math.pi * ic[None, :] * (np.asarray(xc)[:, None] + Lc / 2) / Lc)
    return np.einsum("pi,ji,pj->p", eb, C, ec) / (Nb * Nc)
