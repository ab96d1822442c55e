"""FP64 CPU oracle: discrete adjoint of the PSTD run and of the surface transform.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper has no adjoint; this is the transpose of the oracle's own discrete forward map,
written out step by step so that a reader can check each transpose against the forward
routine it reverses.  Convention: for a real loss L and a complex variable z the gradient is
g_z = dL/dRe z + i dL/dIm z, so that dL = Re(conj(g_z) dz) and a complex-linear map y = M z
pulls back as g_z = M^H g_y.

Forward map (one incidence, EXACT or PAPER form, Eq. PSTDupdating with Eq. expmask):

    u^{n+1} = Gamma [u^{n-1} + A u^n + b^n],   A = -(2 i dt / hbar) (hbar^2/2m eta K + V),

with b^n = -(2 i dt / hbar) V psi_inc^n in the EXACT form (the PAPER form's source does not
depend on V).  K is real symmetric (a circulant with the even eigenvalues k^2), Gamma and V are
real diagonal, so A^H = +(2 i dt / hbar)(hbar^2/2m eta K + V).  The running DFT observes
u^n on the six planes (Eqs. psiphasor, dpsiphasor, scaledphsiphasor, scaleddpsiphasor):

    P_f = (1 / S_f) sum_{n in W} e^{i w_f t_n} E u^n,    S_f = sum_{n in W} e^{i w_f t_n} psi_inc^n(r_O),

E taking psi and the spectral normal derivative on each plane.  Reverse accumulation gives,
with lambda^n the gradient with respect to u^n and mu^n = Gamma lambda^n,

    lambda^n = o^n + A^H mu^{n+1} + mu^{n+2},      o^n = E^H sum_f conj(e^{i w_f t_n} / S_f) g_{P_f},

and, since u^{n+1} depends on V_j through Gamma_j (-(2 i dt / hbar)) (u^n_j + psi_inc^n_j),

    dL/dV_j = sum_n Re[ conj(mu^{n+1}_j) (-(2 i dt / hbar)) (u^n_j + psi_inc^n_j) ]

(without the psi_inc term in the PAPER form, where V multiplies the state alone).
"""
from __future__ import annotations

import math

import numpy as np

from . import ntdf_oracle as no
from .pstd_oracle import FACES, Simulation, apply_axis, kinetic, plane_slice


# ----------------------------------------------------------------------------------
# loss on the Fresnel-region field
# ----------------------------------------------------------------------------------

def magnitude_misfit(psi: np.ndarray, target: np.ndarray):
    """L = sum_p (|psi_p| - target_p)^2 and its gradient g_p = 2 (|psi_p| - target_p) psi_p / |psi_p|."""
    mag = np.abs(psi)
    r = mag - target
    g = 2.0 * r * psi / np.where(mag > 0, mag, 1.0)
    return float(np.sum(r * r)), g


# ----------------------------------------------------------------------------------
# adjoint of the surface transform
# ----------------------------------------------------------------------------------

def transform_adjoint(spec, k: float, points, g_pts):
    """Adjoint of ntdf_oracle.transform_to_points with respect to the six scaled phasor pairs.

    Psi_p is complex-linear in the planes: per face and point it is
    pref * sum_{l,m} e^{ikR}/R [ (A C_d B^T)_{lm} + (ik - 1/R) Rhat_a (A C_p B^T)_{lm} ] with
    C = fft2(plane); so g_C = sum_p conj(coefficient) g_p, and fft2^H = (N_b N_c) ifft2.
    Returns a list of 6 (g_psi_plane, g_dpsi_plane) in the layout of the phasors."""
    pts = np.atleast_2d(np.asarray(points, dtype=float))
    g_pts = np.asarray(g_pts, dtype=np.complex128)
    out = []
    for face in range(6):
        g = no._face_setup(spec, face)
        a, b, c = g["a"], g["b"], g["c"]
        L, M = len(g["cb"]), len(g["cc"])
        Nb, Nc = g["Nb"], g["Nc"]
        pref = -g["sigma"] * g["Db"] * g["Dc"] / (4.0 * math.pi * Nb * Nc)
        gCp = np.zeros((Nc, Nb), dtype=np.complex128)   # gradient w.r.t. C_p[j', i']
        gCd = np.zeros((Nc, Nb), dtype=np.complex128)
        for p, r in enumerate(pts):
            Rb = r[b] - g["cb"][:, None] + 0.0 * g["cc"][None, :]
            Rc = r[c] - g["cc"][None, :] + 0.0 * g["cb"][:, None]
            Ra = np.full((L, M), r[a] - g["plane_coord"])
            R = np.sqrt(Ra * Ra + Rb * Rb + Rc * Rc)
            hb_, hc_, ha_ = Rb / R, Rc / R, Ra / R
            sb = no._usinc(math.pi * g["ib"][None, None, :] / Nb - 0.5 * k * g["Db"] * hb_[:, :, None])
            sc = no._usinc(math.pi * g["ic"][None, None, :] / Nc - 0.5 * k * g["Dc"] * hc_[:, :, None])
            A = (g["eb"][:, None, :] * sb).reshape(L * M, Nb)     # [lm, i']
            B = (g["ec"][None, :, :] * sc).reshape(L * M, Nc)     # [lm, j']
            wd = (pref * np.exp(1j * k * R) / R).reshape(L * M)                  # coefficient of (A C_d B^T)_{lm}
            wp = (pref * np.exp(1j * k * R) / R * (1j * k - 1.0 / R) * ha_).reshape(L * M)
            # S_lm = sum_{i',j'} A[lm,i'] C[j',i'] B[lm,j']  =>  dS_lm/dC[j',i'] = A[lm,i'] B[lm,j']
            gCd += g_pts[p] * np.conj(np.einsum("l,li,lj->ji", wd, A, B))
            gCp += g_pts[p] * np.conj(np.einsum("l,li,lj->ji", wp, A, B))
        out.append((Nb * Nc * np.fft.ifft2(gCp), Nb * Nc * np.fft.ifft2(gCd)))
    return out


# ----------------------------------------------------------------------------------
# adjoint of the leapfrog run
# ----------------------------------------------------------------------------------

def _plane_adjoint(spec, g_face_pairs, coef):
    """E^H applied to coef * (plane gradients): psi parts placed on the planes, normal-
    derivative parts pulled back through the spectral derivative (its adjoint multiplies
    the spectrum by conj(i k))."""
    out = np.zeros(spec.shape, dtype=np.complex128)
    for face, (a, s) in enumerate(FACES):
        h = spec.huygens_lo[a] if s == 0 else spec.huygens_hi[a]
        gp, gd = g_face_pairs[face]
        emb_p = np.zeros(spec.shape, dtype=np.complex128)
        emb_d = np.zeros(spec.shape, dtype=np.complex128)
        plane_slice(emb_p, a, h)[...] = coef * gp
        plane_slice(emb_d, a, h)[...] = coef * gd
        out += emb_p + apply_axis(emb_d, a, spec.d[a], lambda kk: np.conj(1j * kk))
    return out


def forward_states(sim: Simulation, nsteps: int):
    """Run the forward leapfrog, returning u^0 .. u^nsteps (u^0 = 0) and filling the DFT sums."""
    states = [sim.cur.copy()]
    for _ in range(nsteps):
        sim.step(1)
        states.append(sim.cur.copy())
    return states


def adjoint_gradient(sim: Simulation, states, g_phasors):
    """dL/dV (full grid, real) by reverse accumulation, given the forward states u^0..u^N of
    `sim` and g_phasors[f] = the gradient of L with respect to sim.scaled_phasors(f)."""
    spec = sim.spec
    hb = spec.hbar
    c = 2.0 * spec.dt / hb
    nsteps = len(states) - 1

    def AH(x):
        return 1j * c * (sim.kin_coef * kinetic(x, spec.d) + sim.V * x)

    zero = np.zeros(spec.shape, dtype=np.complex128)
    mu1, mu2 = zero, zero            # mu^{n+1}, mu^{n+2}
    grad = np.zeros(spec.shape)
    for n in range(nsteps, -1, -1):
        # V enters u^{n+1} (n <= N - 1) through Gamma (-(i c)) (u^n + psi_inc^n)
        if n <= nsteps - 1:
            base = states[n] + (sim.psi_inc(n) if spec.tfsf_mode == "exact" else 0.0)
            grad += np.real(np.conj(mu1) * (-1j * c) * base)
        lam = AH(mu1) + mu2
        if sim.in_window(n):
            t = n * spec.dt
            for fi, w in enumerate(sim.omegas):
                coef = np.conj(complex(math.cos(w * t), math.sin(w * t)) / sim.acc_inc[fi])
                lam = lam + _plane_adjoint(spec, g_phasors[fi], coef)
        mu2, mu1 = mu1, sim.Gamma * lam
    return grad


def fresnel_loss_and_gradient(spec, V, khat, k, ramp_time, window, nsteps, points, target, omega=None):
    """L(V) = sum_p (|Psi_p| - target_p)^2 for the Fresnel field of the scaled phasors at one
    frequency (default the carrier), and dL/dV by the discrete adjoint.  Returns (L, grad, psi)."""
    sim = Simulation(spec, V, khat, k, ramp_time, window=window, omegas=None if omega is None else [omega])
    states = forward_states(sim, nsteps)
    ph = sim.scaled_phasors(0)
    psi = no.transform_to_points(spec, k, ph, points)
    L, g_pts = magnitude_misfit(psi, target)
    g_ph = transform_adjoint(spec, k, points, g_pts)
    grad = adjoint_gradient(sim, states, [g_ph])
    return L, grad, psi


def fresnel_loss(spec, V, khat, k, ramp_time, window, nsteps, points, target, omega=None) -> float:
    """The loss alone (forward run only), for finite differences."""
    sim = Simulation(spec, V, khat, k, ramp_time, window=window, omegas=None if omega is None else [omega])
    sim.step(nsteps)
    psi = no.transform_to_points(spec, k, sim.scaled_phasors(0), points)
    return magnitude_misfit(psi, target)[0]
