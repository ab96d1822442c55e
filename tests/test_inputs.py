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
