"""Pins of the spinor oracle (CPU).

For B(r) = b(r) nhat with a fixed direction nhat, sigma . B = b(r) sigma . nhat has constant
eigenvectors e+, e- (eigenvalues +-1), so the spinor problem splits exactly into two scalar
problems with potentials V +- gamma b(r): an incident spin state chi = a e+ + c e- scatters into
u = a e+ u+ + c e- u-, with u+- the scalar oracle's runs.  This pins the diagonal (nhat = z)
and the spin-flip (nhat = x, y, oblique) couplings, their signs and the complex i By terms,
against the pinned scalar oracle.  A planted sign error in By must break the pin.
"""
import math

import numpy as np
import pytest

from oracle import pstd_oracle as po
from oracle import spinor_oracle as so
from paper_2403_04053_gb300 import inputs

K = 2 * math.pi
KHAT = (0.3, -0.5, 0.81)


def spec():
    return inputs.GridSpec(n=(24, 24, 24), d=(0.25, 0.25, 0.25), dt=0.003, abc_cells=(3, 3, 3), tfsf_lo=(6, 6, 6),
                           tfsf_hi=(17, 17, 17), taper_cells=2, huygens_lo=(4, 4, 4), huygens_hi=(19, 19, 19))


def fields(sp, nhat, seed=3):
    rng = np.random.default_rng(seed)
    x = [sp.coords(a) for a in range(3)]
    Z, Y, X = np.meshgrid(x[2], x[1], x[0], indexing="ij")
    c = sp.core_box()
    inside = np.zeros(sp.shape, bool)
    inside[c[2][0]:c[2][1] + 1, c[1][0]:c[1][1] + 1, c[0][0]:c[0][1] + 1] = True
    V = np.where(inside, rng.uniform(-2, 2, sp.shape), 0.0)
    b = np.where(inside, 4.0 * np.exp(-(X ** 2 + Y ** 2 + Z ** 2) / 2.0), 0.0)
    n = np.asarray(nhat, float) / np.linalg.norm(nhat)
    return V, (b * n[0], b * n[1], b * n[2]), b


@pytest.mark.parametrize("nhat", [(0, 0, 1), (1, 0, 0), (0, 1, 0), (0.3, -0.6, 0.74)])
def test_spinor_splits_into_scalar_problems(nhat):
    sp = spec()
    gamma = 1.7
    V, B, b = fields(sp, nhat)
    chi = (0.6, 0.8j)
    win = (20, 20)
    sim = so.SpinorSimulation(sp, V, B, gamma, KHAT, K, 0.05, chi, window=win)
    sim.step(40)
    ep, em = so.eigen_spin(np.asarray(nhat, float) / np.linalg.norm(nhat))
    a, c = np.vdot(ep, chi), np.vdot(em, chi)          # chi = a e+ + c e-
    up = po.Simulation(sp, V + gamma * b, KHAT, K, 0.05, window=win)
    dn = po.Simulation(sp, V - gamma * b, KHAT, K, 0.05, window=win)
    up.step(40)
    dn.step(40)
    for s in range(2):
        ref = a * ep[s] * up.cur + c * em[s] * dn.cur
        assert np.linalg.norm(sim.cur[s] - ref) <= 1e-12 * np.linalg.norm(ref)
        for face in range(6):
            for q in range(2):
                r = a * ep[s] * up.scaled_phasors(0)[face][q] + c * em[s] * dn.scaled_phasors(0)[face][q]
                assert np.linalg.norm(sim.scaled_phasors(s)[face][q] - r) <= 1e-11 * np.linalg.norm(r) + 1e-300


def test_planted_by_sign_error_is_caught(monkeypatch):
    sp = spec()
    V, B, b = fields(sp, (0, 1, 0))

    def wrong(V_, B_, gamma):
        Bx, By, Bz = B_
        return (V_ + gamma * Bz, gamma * (Bx + 1j * By), gamma * (Bx - 1j * By), V_ - gamma * Bz)
    monkeypatch.setattr(so, "coupling", wrong)
    chi = (1.0, 0.0)
    sim = so.SpinorSimulation(sp, V, B, 1.7, KHAT, K, 0.05, chi)
    sim.step(30)
    ep, em = so.eigen_spin((0.0, 1.0, 0.0))
    a, c = np.vdot(ep, chi), np.vdot(em, chi)
    up = po.Simulation(sp, V + 1.7 * b, KHAT, K, 0.05)
    dn = po.Simulation(sp, V - 1.7 * b, KHAT, K, 0.05)
    up.step(30)
    dn.step(30)
    ref = a * ep[1] * up.cur + c * em[1] * dn.cur
    assert np.linalg.norm(sim.cur[1] - ref) > 1e-3 * np.linalg.norm(ref)


def test_node_sampled_step_equals_whole_array_step():
    # the node-by-node update (three grid lines per node) against the whole-array step, on nodes
    # in the absorber, at the grid's edges, in the taper and inside B's support
    sp = spec()
    V, B, _ = fields(sp, (0.3, -0.6, 0.74))
    rng = np.random.default_rng(9)
    B = [b + np.where(b != 0, rng.uniform(-1, 1, sp.shape), 0.0) for b in B]     # a varying direction
    prev = [inputs.random_field(sp.shape, 20 + s) for s in range(2)]
    cur = [inputs.random_field(sp.shape, 22 + s) for s in range(2)]
    gamma, chi = 1.3, (0.6, 0.8j)
    sim = so.SpinorSimulation(sp, V, B, gamma, KHAT, K, 0.05, chi)
    for s in range(2):
        sim.comp[s].prev, sim.comp[s].cur, sim.comp[s].n = prev[s].copy(), cur[s].copy(), 9
    sim.n = 9
    sim.step(1)
    nodes = [(0, 0, 0), (23, 23, 23), (1, 12, 22), (7, 8, 9), (12, 12, 12), (11, 13, 10)]
    nodes += [tuple(int(v) for v in rng.integers(0, 24, 3)) for _ in range(40)]
    got = so.step_at_nodes(sp, V, B, gamma, KHAT, K, 0.05, chi, prev, cur, 9, nodes)
    for q, (i, j, k) in enumerate(nodes):
        for s in range(2):
            assert abs(got[q, s] - sim.cur[s][k, j, i]) <= 1e-12 * (1 + abs(sim.cur[s][k, j, i]))
