"""Pins of the oracle's discrete adjoint (CPU).

The gradient of the Fresnel-field misfit with respect to V is checked against central
finite differences of the oracle's own forward loss, which is the definition of the
derivative, and the adjoint of the surface transform against the transpose identity
Re<T x, y> = Re<x, T^H y>.  A planted sign error in the adjoint's kinetic operator must
make the finite-difference pin fail.
"""
import math

import numpy as np
import pytest

from oracle import adjoint_oracle as ao
from oracle import ntdf_oracle as no
from oracle import pstd_oracle as po
from paper_2403_04053_gb300 import inputs

K = 2 * math.pi
KHAT = (0.3, -0.5, 0.81)
PTS = np.array([[3.0, -2.0, 5.5], [-4.0, 6.0, 1.0], [0.5, 0.2, -9.0], [1.0, 2.0, 3.0]])


def small_spec(mode):
    return inputs.GridSpec(n=(24, 24, 24), d=(0.25, 0.25, 0.25), dt=0.004, abc_cells=(3, 3, 3), tfsf_lo=(6, 6, 6),
                           tfsf_hi=(17, 17, 17), taper_cells=2, huygens_lo=(4, 4, 4), huygens_hi=(19, 19, 19),
                           tfsf_mode=mode)


def core_V(spec, seed):
    rng = np.random.default_rng(seed)
    V = np.zeros(spec.shape)
    c = spec.core_box()
    sl = (slice(c[2][0], c[2][1] + 1), slice(c[1][0], c[1][1] + 1), slice(c[0][0], c[0][1] + 1))
    V[sl] = rng.uniform(-3, 3, V[sl].shape)
    return V


def _fd_check(spec, V, grad, voxels, h=1e-4):
    args = (KHAT, K, 0.05, (50, 30), 80, PTS, np.full(len(PTS), 0.01))
    errs = []
    for (z, y, x) in voxels:
        Vp, Vm = V.copy(), V.copy()
        Vp[z, y, x] += h
        Vm[z, y, x] -= h
        fd = (ao.fresnel_loss(spec, Vp, *args) - ao.fresnel_loss(spec, Vm, *args)) / (2 * h)
        errs.append(abs(fd - grad[z, y, x]))
    return max(errs) / np.abs(grad).max()


@pytest.mark.parametrize("mode", ["exact", "paper"])
def test_adjoint_gradient_matches_central_differences(mode):
    spec = small_spec(mode)
    V = core_V(spec, 7)
    L, grad, psi = ao.fresnel_loss_and_gradient(spec, V, KHAT, K, 0.05, (50, 30), 80, PTS, np.full(len(PTS), 0.01))
    assert L > 0 and np.abs(grad).max() > 0
    rng = np.random.default_rng(11)
    inside = np.argwhere(V != 0)
    voxels = [tuple(v) for v in inside[rng.choice(len(inside), 6, replace=False)]]
    if mode == "exact":
        voxels.append((2, 12, 12))             # V = 0 there; the EXACT form allows V anywhere
    assert _fd_check(spec, V, grad, voxels) < 1e-6


def test_planted_adjoint_sign_error_is_caught(monkeypatch):
    spec = small_spec("exact")
    V = core_V(spec, 7)
    monkeypatch.setattr(ao, "kinetic", lambda u, d: -po.kinetic(u, d))   # A in place of A^H for K
    L, grad, psi = ao.fresnel_loss_and_gradient(spec, V, KHAT, K, 0.05, (50, 30), 80, PTS, np.full(len(PTS), 0.01))
    inside = np.argwhere(V != 0)
    assert _fd_check(spec, V, grad, [tuple(v) for v in inside[:3]]) > 1e-2


def test_transform_adjoint_is_the_transpose():
    spec = small_spec("exact")
    rng = np.random.default_rng(3)
    x = []
    for face, (a, s) in enumerate(po.FACES):
        shp = po.plane_slice(np.zeros(spec.shape), a, 0).shape
        x.append(tuple(rng.standard_normal(shp) + 1j * rng.standard_normal(shp) for _ in range(2)))
    y = rng.standard_normal(len(PTS)) + 1j * rng.standard_normal(len(PTS))
    Tx = no.transform_to_points(spec, K, x, PTS)
    THy = ao.transform_adjoint(spec, K, PTS, y)
    lhs = np.vdot(y, Tx)
    rhs = sum(np.vdot(THy[f][q], x[f][q]) for f in range(6) for q in range(2))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_plane_adjoint_is_the_transpose():
    # E u: psi and the spectral normal derivative on the six planes; E^H from the adjoint module
    spec = small_spec("exact")
    rng = np.random.default_rng(5)
    u = rng.standard_normal(spec.shape) + 1j * rng.standard_normal(spec.shape)
    Eu = []
    for face, (a, s) in enumerate(po.FACES):
        h = spec.huygens_lo[a] if s == 0 else spec.huygens_hi[a]
        Eu.append((po.plane_slice(u, a, h), po.plane_slice(po.derivative(u, a, spec.d[a]), a, h)))
    y = [tuple(rng.standard_normal(p.shape) + 1j * rng.standard_normal(p.shape) for p in pair) for pair in Eu]
    EHy = ao._plane_adjoint(spec, y, 1.0)
    lhs = sum(np.vdot(y[f][q], Eu[f][q]) for f in range(6) for q in range(2))
    rhs = np.vdot(EHy, u)
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)
