"""Pins of the oracle's near-to-distant-field transform (Section 3) against closed forms.

CPU only.  The transform is checked on analytic surface data: an outgoing spherical
wave must be reproduced outside the virtual box and vanish inside it (the surface
equivalence theorem, Eqs. P, PsiDF, surfequivtheorem), its far-field amplitude is a
pure phase, a source-free plane wave gives nothing outside, and the paper's per-cell
sinc sum equals a brute-force quadrature of the cell integral it stands for.
"""
import math

import numpy as np
import pytest

from oracle import analytic as an
from oracle import ntdf_oracle as no
from oracle import pstd_oracle as po
from paper_2403_04053_gb300 import inputs

K = 2 * math.pi


def _spec(n=48, d=0.25, hb=(11, 37)):
    return inputs.GridSpec(n=(n, n, n), d=(d, d, d), dt=0.004, huygens_lo=(hb[0],) * 3, huygens_hi=(hb[1],) * 3)


def _window(n, lo, hi):
    """1 on [lo, hi], a smooth (xi-shaped) fall to 0 over the `lo` cells outside, 0 beyond."""
    i = np.arange(n, dtype=float)
    w = np.ones(n)
    r = np.clip(i / lo, 0, 1)
    w = np.where(i < lo, po.xi(r), w)
    r = np.clip((n - 1 - i) / (n - 1 - hi), 0, 1)
    w = np.where(i > hi, po.xi(r), w)
    return w


def field_planes(spec, field_fn, margin=3):
    """Six (psi, d psi / d a) plane pairs of an analytic field, windowed to 0 at the plane edges
    (the absorbing layer's role in Section 3.3) and exact over the virtual surface."""
    out = []
    for face, (a, s) in enumerate(po.FACES):
        b, c = po.in_plane_axes(a)
        h = spec.huygens_lo[a] if s == 0 else spec.huygens_hi[a]
        xb, xc = po.coords(spec.n[b], spec.d[b]), po.coords(spec.n[c], spec.d[c])
        XC, XB = np.meshgrid(xc, xb, indexing="ij")
        pts = np.zeros(XB.shape + (3,))
        pts[..., a] = po.coords(spec.n[a], spec.d[a])[h]
        pts[..., b] = XB
        pts[..., c] = XC
        psi, grad = field_fn(pts.reshape(-1, 3))
        wb = _window(spec.n[b], spec.huygens_lo[b] - margin, spec.huygens_hi[b] + margin)
        wc = _window(spec.n[c], spec.huygens_lo[c] - margin, spec.huygens_hi[c] + margin)
        W = wc[:, None] * wb[None, :]
        out.append((W * psi.reshape(XB.shape), W * grad[:, a].reshape(XB.shape)))
    return out


def _sph(src):
    return lambda p: an.spherical_wave(p, K, src)


@pytest.fixture(scope="module")
def sph_planes():
    spec = _spec()
    src = (0.3, -0.2, 0.45)
    return spec, src, field_planes(spec, _sph(src))


def test_spherical_wave_is_reproduced_outside_the_box(sph_planes):
    """Exterior points at 2..60 box half-widths: Psi = e^{ik rho}/rho (the paper's NTDF validation, Section 3.4)."""
    spec, src, ph = sph_planes
    rng = np.random.default_rng(3)
    dirs = rng.standard_normal((12, 3))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    for r, tol in [(8.0, 1.5e-2), (30.0, 3e-3), (200.0, 1.5e-3)]:
        pts = dirs * r
        got = no.transform_to_points(spec, K, ph, pts)
        ref, _ = an.spherical_wave(pts, K, src)
        err = np.abs(got - ref) / np.abs(ref)
        assert np.max(err) < tol, (r, np.max(err))


def test_spherical_wave_vanishes_inside_the_box(sph_planes):
    """Psi_DF = P Psi = 0 inside V (Eqs. P, PsiDF)."""
    spec, src, ph = sph_planes
    pts = np.array([[1.0, 1.2, -0.7], [-2.0, 0.5, 1.5], [0.0, -1.8, -2.2]])
    got = no.transform_to_points(spec, K, ph, pts)
    ref, _ = an.spherical_wave(pts, K, src)
    assert np.max(np.abs(got) / np.abs(ref)) < 3e-3


def test_far_field_of_a_spherical_wave_is_a_pure_phase(sph_planes):
    """f(rhat) = e^{-ik rhat . r_s} exactly for e^{ik|r - r_s|}/|r - r_s|; dsigma/dOmega = 1."""
    spec, src, ph = sph_planes
    th = np.deg2rad(np.arange(0, 181, 10.0))
    phi = np.deg2rad(np.linspace(0, 330, len(th)))
    ds, f = no.cross_section(spec, K, ph, th, phi)
    rh = np.stack([np.sin(th) * np.cos(phi), np.sin(th) * np.sin(phi), np.cos(th)], axis=1)
    ref = np.exp(-1j * K * rh @ np.asarray(src))
    assert np.max(np.abs(f - ref)) < 1e-3
    assert np.max(np.abs(ds - 1.0)) < 2e-3


def test_plane_wave_data_give_nothing_outside():
    """A source-free incident plane wave contributes 0 to the exterior field (the point of feeding only the
    scattered field to the surface integral)."""
    spec = _spec()
    kv = K * np.array([0.36, 0.48, 0.8])

    def pw(p):
        psi = np.exp(1j * p @ kv)
        return psi, 1j * psi[:, None] * kv[None, :]

    ph = field_planes(spec, pw)
    pts = np.array([[0, 0, 20.0], [15.0, -3.0, 4.0], [-5.0, 30.0, -8.0]])
    assert np.max(np.abs(no.transform_to_points(spec, K, ph, pts))) < 2e-3 * 1.0


def test_sign_of_the_face_term_is_pinned(sph_planes, monkeypatch):
    """Planted mistake: flipping the outward-normal sign of one face breaks the spherical-wave pin."""
    spec, src, ph = sph_planes
    orig = no._face_setup

    def bad(spec_, face):
        g = orig(spec_, face)
        if face == 4:
            g["sigma"] = -g["sigma"]
        return g

    monkeypatch.setattr(no, "_face_setup", bad)
    pts = np.array([[0.0, 0.0, 30.0], [0.0, 0.0, -30.0]])
    got = no.transform_to_points(spec, K, ph, pts)
    ref, _ = an.spherical_wave(pts, K, src)
    assert np.max(np.abs(got - ref) / np.abs(ref)) > 0.1


def test_per_cell_sinc_sum_equals_quadrature_of_the_cell_integral():
    """The closed-form sinc sum of Eq. bottomPsi_lm = a 16x16 Gauss-Legendre quadrature of
    -sigma/(4 pi) e^{ikR}/R * int_cell [d psi_an + (ik - 1/R) Rhat_a psi_an] e^{-ik Rhat . dr'} dS',
    with psi_an evaluated from its definition (Eq. AnBottomPsi); random band-limited plane data."""
    n = 12
    spec = inputs.GridSpec(n=(n, n, n), d=(0.25, 0.3, 0.2), dt=0.004, huygens_lo=(3, 4, 2), huygens_hi=(9, 8, 10))
    rng = np.random.default_rng(11)
    ph = []
    for face, (a, s) in enumerate(po.FACES):
        b, c = po.in_plane_axes(a)
        shape = (spec.n[c], spec.n[b])
        ph.append((rng.standard_normal(shape) + 1j * rng.standard_normal(shape),
                   rng.standard_normal(shape) + 1j * rng.standard_normal(shape)))
    pts = np.array([[4.0, -3.0, 2.5], [-1.0, 0.5, 6.0]])
    got = no.transform_to_points(spec, K, ph, pts)
    gx, gw = np.polynomial.legendre.leggauss(16)
    ref = np.zeros(len(pts), dtype=complex)
    for face, (a, s) in enumerate(po.FACES):
        b, c = po.in_plane_axes(a)
        sigma = -1.0 if s == 0 else 1.0
        h = spec.huygens_lo[a] if s == 0 else spec.huygens_hi[a]
        za = po.coords(spec.n[a], spec.d[a])[h]
        Db, Dc = spec.d[b], spec.d[c]
        xb, xc = po.coords(spec.n[b], Db), po.coords(spec.n[c], Dc)
        for l in range(spec.huygens_lo[b], spec.huygens_hi[b]):
            for m in range(spec.huygens_lo[c], spec.huygens_hi[c]):
                cb, cc = xb[l] + Db / 2, xc[m] + Dc / 2
                qb = (cb + 0.5 * Db * gx)[:, None] + 0 * gx[None, :]
                qc = (cc + 0.5 * Dc * gx)[None, :] + 0 * gx[:, None]
                wq = np.outer(gw, gw) * 0.25 * Db * Dc
                psi = no.interpolant(ph[face][0], spec.n[b], spec.n[c], Db, Dc, qb.ravel(), qc.ravel())
                dps = no.interpolant(ph[face][1], spec.n[b], spec.n[c], Db, Dc, qb.ravel(), qc.ravel())
                for p, r in enumerate(pts):
                    Rv = np.zeros(3)
                    Rv[a], Rv[b], Rv[c] = r[a] - za, r[b] - cb, r[c] - cc
                    R = np.linalg.norm(Rv)
                    Rh = Rv / R
                    lin = np.exp(-1j * K * (Rh[b] * (qb.ravel() - cb) + Rh[c] * (qc.ravel() - cc)))
                    integ = np.sum(wq.ravel() * (dps + (1j * K - 1 / R) * Rh[a] * psi) * lin)
                    ref[p] += -sigma / (4 * math.pi) * np.exp(1j * K * R) / R * integ
    assert np.max(np.abs(got - ref)) < 1e-11 * np.max(np.abs(ref))
