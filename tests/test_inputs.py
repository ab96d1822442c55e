"""Checks of the seeded workload generators (inputs only; no method arithmetic)."""
import math

import numpy as np

from paper_2403_04053_gb300 import inputs


def test_voxelised_sphere_has_the_sphere_volume():
    wl = inputs.square_barrier_workload(with_outputs=False)
    V0 = 0.3 * 2 * math.pi ** 2
    vol = wl.V.sum() / V0 * 0.25 ** 3
    assert abs(vol - 4.0 / 3.0 * math.pi * 1.5 ** 3) < 0.01 * vol


def test_gaussian_sum_is_seeded_and_confined_to_the_core():
    spec = inputs.gaussian_sum_workload(n=64, tf=(12, 52), hb=(10, 54), abc=8, with_outputs=False).spec
    a = inputs.gaussian_sum_potential(spec, 19.7, seed=3)
    b = inputs.gaussian_sum_potential(spec, 19.7, seed=3)
    assert np.array_equal(a, b)
    core = spec.core_box()
    mask = np.zeros(spec.shape, dtype=bool)
    mask[core[2][0]:core[2][1] + 1, core[1][0]:core[1][1] + 1, core[0][0]:core[0][1] + 1] = True
    assert np.count_nonzero(a[~mask]) == 0 and np.count_nonzero(a[mask]) > 0


def test_fibonacci_directions_are_unit_and_spread():
    d = inputs.fibonacci_directions(8)
    assert np.allclose(np.linalg.norm(d, axis=1), 1.0)
    assert np.abs(d.mean(axis=0)).max() < 0.2


def test_dipole_field_formula_window_and_divergence():
    # a small grid holding r <= 12 with the same spacing as the 384^3 workload
    spec = inputs.GridSpec(n=(128, 128, 128), d=(0.25,) * 3, dt=1.0, abc_cells=(4,) * 3, tfsf_lo=(8,) * 3,
                           tfsf_hi=(120,) * 3, taper_cells=2, huygens_lo=(6,) * 3, huygens_hi=(122,) * 3)
    m = np.array([0.3, -0.4, 0.866])
    m /= np.linalg.norm(m)
    B = inputs.dipole_field(spec, m)
    x = spec.coords(0)
    # inside the plateau 1 <= r <= 11 the field is (3 (m . rhat) rhat - m) / r^3
    for (i, j, k) in [(64 + 12, 64, 64), (64, 64 - 20, 64 + 8), (64 + 7, 64 + 7, 64 - 7)]:
        r = np.array([x[i], x[j], x[k]])
        rn = np.linalg.norm(r)
        ref = (3 * (m @ r) * r / rn ** 2 - m) / rn ** 3
        assert np.allclose([B[a][k, j, i] for a in range(3)], ref, rtol=1e-12, atol=0)
    # zero inside r <= 1/2 and outside r >= 12
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    R = np.sqrt(X * X + Y * Y + Z * Z)
    mag = np.sqrt(B[0] ** 2 + B[1] ** 2 + B[2] ** 2)
    assert not np.any(mag[(R <= 0.5) | (R >= 12.0)])
    # divergence-free on the plateau (central differences of a smooth field, h = 0.25)
    h = 0.25
    div = ((B[0][:, :, 2:] - B[0][:, :, :-2])[1:-1, 1:-1, :] + (B[1][:, 2:, :] - B[1][:, :-2, :])[1:-1, :, 1:-1]
           + (B[2][2:, :, :] - B[2][:-2, :, :])[:, 1:-1, 1:-1]) / (2 * h)
    Rc = R[1:-1, 1:-1, 1:-1]
    plateau = (Rc >= 3.0) & (Rc <= 10.0)
    scale = mag[1:-1, 1:-1, 1:-1][plateau].max() / h
    assert np.max(np.abs(div[plateau])) < 0.05 * scale


def test_spinor_workload_geometry_and_strength():
    # a 128^3 grid whose zeta = 1 core (12..116, |x| <= 13) holds the r <= 12 support
    wl = inputs.spinor_workload(n=128, tf=(8, 120), hb=(6, 122), abc=4, nsteps=400, with_outputs=False)
    sp = wl.spec
    E = 0.5 * (2 * math.pi) ** 2
    mag = np.sqrt(wl.B[0] ** 2 + wl.B[1] ** 2 + wl.B[2] ** 2)
    assert abs(wl.gamma * mag.max() - 0.5 * E) < 1e-9 * E
    core = sp.core_box()
    inside = np.zeros(sp.shape, dtype=bool)
    inside[core[2][0]:core[2][1] + 1, core[1][0]:core[1][1] + 1, core[0][0]:core[0][1] + 1] = True
    assert not np.any(mag[~inside])
    # dt = 0.9 x the bound with |gamma B|max (Eq. PSTDstability, hbar = m = 1)
    kin = 0.5 * math.pi ** 2 * sum(1.0 / d ** 2 for d in sp.d)
    assert abs(sp.dt - 0.9 / (kin + 0.5 * E)) < 1e-15
    assert wl.chis == [(1.0, 0.0), (0.0, 1.0)] and not np.any(wl.V)
