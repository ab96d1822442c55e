"""GPU parity of the 1-D auxiliary incident wave (pstd_set_incidence_aux, Section 2.2.3) against
the FP64 oracle (oracle/aux_oracle.py driving pstd_oracle.Simulation).

Tolerances: those of the CW path, FP64 1e-12 after one step and FP32 2e-6. The evaluated
incident wave adds at most 32 + nm/32 rounded complex products per term in FP32 (here nm <= 256,
so < 40 * 6e-8 of |psi_inc|), which enters the state multiplied by 2 dt V / hbar.
"""
import math

import numpy as np
import pytest

from oracle import aux_oracle as ao
from oracle import ntdf_oracle as no
from oracle import pstd_oracle as po
from paper_2403_04053_gb300 import inputs, pstd

pytestmark = pytest.mark.gpu

K = 2 * math.pi
E0 = 0.5 * K * K
KHAT = (0.3, -0.5, 0.81)
AXIS = (-4.0, 0.125, 256)          # d_lo, dd, n1: covers the ragged grid's TF/SF box (d <= 4.1)


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def ragged_spec(mode="exact"):
    return inputs.GridSpec(n=(24, 32, 48), d=(0.25, 0.3, 0.2), dt=0.002, abc_cells=(4, 5, 6), tfsf_lo=(9, 12, 17),
                           tfsf_hi=(15, 20, 31), taper_cells=2, huygens_lo=(7, 9, 14), huygens_hi=(17, 23, 34),
                           tfsf_mode=mode)


def random_core_V(spec, seed, amp=3.0):
    rng = np.random.default_rng(seed)
    V = np.zeros(spec.shape)
    c = spec.core_box()
    V[c[2][0]:c[2][1] + 1, c[1][0]:c[1][1] + 1, c[0][0]:c[0][1] + 1] = rng.uniform(
        -amp, amp, (c[2][1] - c[2][0] + 1, c[1][1] - c[1][0] + 1, c[0][1] - c[0][0] + 1))
    return V


def axis_d():
    d_lo, dd, n1 = AXIS
    return d_lo + dd * np.arange(n1)


def gaussian_profile(sigma=0.6, d0=-1.0):
    return po.gaussian_packet(axis_d() - d0, 0.0, K, sigma)


def random_profile(seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal(AXIS[2]) + 1j * rng.standard_normal(AXIS[2])


def oracle_aux(spec, profile):
    return ao.AuxSource1D(AXIS[0], AXIS[1], profile, E0, spec.dt)


@pytest.mark.parametrize("prec,tol", [(pstd.F64, 1e-12), (pstd.F32, 2e-6)])
@pytest.mark.parametrize("mode", ["exact", "paper"])
def test_one_step_matches_oracle(mode, prec, tol):
    # a random profile: every mode of the 256-point axis is active
    spec = ragged_spec(mode)
    V = random_core_V(spec, 3)
    prof = random_profile(8)
    prev = inputs.random_field(spec.shape, 5)
    cur = inputs.random_field(spec.shape, 6)
    sim = po.Simulation(spec, V, KHAT, K, 0.0, aux=oracle_aux(spec, prof))
    sim.prev, sim.cur, sim.n = prev.copy(), cur.copy(), 17
    sim.step(1)
    cd = np.complex128 if prec == pstd.F64 else np.complex64
    with pstd.Grid(spec, precision=prec) as g:
        g.set_potential(V)
        g.set_incidence_aux(0, KHAT, K, AXIS[0], AXIS[1], prof)
        g.set_field(0, prev.astype(cd), cur.astype(cd), 17)
        g.step(1)
        assert rel(g.get_field(0), sim.cur) < tol


@pytest.mark.parametrize("prec,tol_state,tol_out", [(pstd.F64, 1e-12, 1e-10), (pstd.F32, 2e-5, 2e-4)])
@pytest.mark.parametrize("mode", ["exact", "paper"])
def test_packet_run_phasors_transform_far_field(mode, prec, tol_state, tol_out):
    # a Gaussian profile through the auxiliary wave: 60 steps, 40 in the window, 3 frequencies
    spec = ragged_spec(mode)
    V = random_core_V(spec, 1)
    om = [0.9 * E0, E0, 1.1 * E0]
    sim = po.Simulation(spec, V, KHAT, K, 0.0, window=(20, 40), omegas=om, aux=oracle_aux(spec, gaussian_profile()))
    sim.step(60)
    pts = np.array([[3.0, -2.0, 5.5], [-4.0, 6.0, 1.0], [30.0, 10.0, 40.0]])
    th, ph = np.deg2rad([5.0, 91.0, 170.0]), np.deg2rad([10.0, 250.0, 0.0])
    with pstd.Grid(spec, precision=prec) as g:
        g.set_potential(V)
        g.set_incidence_aux(0, KHAT, K, AXIS[0], AXIS[1], gaussian_profile())
        g.huygens_dft(0, om, 20, 40)
        g.step(60)
        assert rel(g.get_field(0), sim.cur) < tol_state
        if mode == "paper":
            assert rel(g.get_field(0, pstd.FIELD_SCATTERED), sim.scattered_field()) < tol_state
        for f in range(3):
            ref = sim.scaled_phasors(f)
            for a, b in zip(g.get_phasors(0, f), ref):
                assert rel(a[0], b[0]) < 10 * tol_state and rel(a[1], b[1]) < 10 * tol_state
            kf = math.sqrt(2 * om[f])
            assert rel(g.transform_to_points(0, f, pts), no.transform_to_points(spec, kf, ref, pts)) < tol_out
            _, fref = no.cross_section(spec, kf, ref, th, ph)
            assert rel(g.cross_section(0, f, th, ph)[1], fref) < tol_out


@pytest.mark.parametrize("mode", ["exact", "paper"])
def test_carrier_mode_profile_equals_the_cw_run(mode):
    # e^{i k d} on an axis holding k: the 1-D scheme's root at the carrier is e^{-i E dt}, so the
    # run equals the CW run without a ramp
    spec = ragged_spec(mode)
    V = random_core_V(spec, 4)
    prof = np.exp(1j * K * axis_d())
    out = []
    for aux in (False, True):
        with pstd.Grid(spec, precision=pstd.F64) as g:
            g.set_potential(V)
            if aux:
                g.set_incidence_aux(0, KHAT, K, AXIS[0], AXIS[1], prof)
            else:
                g.set_incidence(0, KHAT, K, 0.0)
            g.huygens_dft(0, [E0], 10, 20)
            g.step(40)
            out.append((g.get_field(0), g.join_phasors(g.get_phasors(0, 0))))
    assert rel(out[1][0], out[0][0]) < 1e-11
    assert rel(out[1][1], out[0][1]) < 1e-10


def test_aux_and_cw_members_in_one_batch_equal_separate_runs():
    spec = ragged_spec()
    V = random_core_V(spec, 2)
    prof = gaussian_profile()

    def setup(g, b, aux):
        if aux:
            g.set_incidence_aux(b, KHAT, K, AXIS[0], AXIS[1], prof)
        else:
            g.set_incidence(b, (-0.6, 0.0, 0.8), K, 0.05)
        g.huygens_dft(b, [E0], 10, 20)

    single = []
    for aux in (True, False):
        with pstd.Grid(spec, precision=pstd.F32) as g:
            g.set_potential(V)
            setup(g, 0, aux)
            g.step(30)
            single.append((g.get_field(0), g.join_phasors(g.get_phasors(0, 0))))
    with pstd.Grid(spec, precision=pstd.F32, batch=3) as g:
        g.set_potential(V)
        setup(g, 0, False)
        setup(g, 1, True)
        setup(g, 2, False)
        g.step(30)
        assert np.array_equal(g.get_field(1), single[0][0])
        assert np.array_equal(g.join_phasors(g.get_phasors(1, 0)), single[0][1])
        for b in (0, 2):
            assert np.array_equal(g.get_field(b), single[1][0])
        # switching member 1 back to CW drops its auxiliary wave
        g.reset()
        setup(g, 1, False)
        g.step(30)
        assert np.array_equal(g.get_field(1), single[1][0])


def test_graph_replay_with_an_aux_member():
    spec = ragged_spec("paper")
    V = random_core_V(spec, 6)
    res = []
    for graphs in (False, True):
        with pstd.Grid(spec, precision=pstd.F32) as g:
            g.set_graphs(graphs)
            g.set_potential(V)
            g.set_incidence_aux(0, KHAT, K, AXIS[0], AXIS[1], gaussian_profile())
            g.huygens_dft(0, [E0], 5, 10)
            for _ in range(3):
                g.reset()
                g.step(20)
            res.append((g.get_field(0), g.join_phasors(g.get_phasors(0, 0)), g.graph_replays()))
    assert res[0][2] == 0 and res[1][2] == 2
    assert np.array_equal(res[0][0], res[1][0]) and np.array_equal(res[0][1], res[1][1])


def test_aux_call_errors():
    spec = ragged_spec()
    prof = gaussian_profile()
    with pstd.Grid(spec, precision=pstd.F32) as g:
        cases = [((AXIS[0], AXIS[1], prof[:200]), "EINVAL"),                     # n1 not a power of two
                 ((0.5, AXIS[1], prof), "EINVAL"),                               # the axis starts inside the box
                 ((-30.0, AXIS[1], prof[:128]), "EINVAL"),                       # ... and ends before its far side
                 ((AXIS[0], 0.02, np.ones(1024)), "EUNSTABLE")]                  # too fine for dt
        for (d_lo, dd, p), code in cases:
            with pytest.raises(pstd.PstdError) as e:
                g.set_incidence_aux(0, KHAT, K, d_lo, dd, p)
            assert e.value.code == code
        bad = prof.copy()
        bad[3] = np.nan
        with pytest.raises(pstd.PstdError) as e:
            g.set_incidence_aux(0, KHAT, K, AXIS[0], AXIS[1], bad)
        assert e.value.code == "EINVAL"
        # the adjoint runs CW members only
        g.set_potential(random_core_V(spec, 1))
        g.set_incidence_aux(0, KHAT, K, AXIS[0], AXIS[1], prof)
        g.huygens_dft(0, [E0], 10, 20)
        g.step(30)
        with pytest.raises(pstd.PstdError) as e:
            g.adjoint_gradient(30, [np.ones(g.phasor_count(), complex)], (11, 14, 19), (13, 18, 29))
        assert e.value.code == "EINVAL"
    with pstd.Grid(spec, precision=pstd.F32, batch=2) as g:                      # spinor grids
        V = random_core_V(spec, 1)
        g.set_magnetic_field([V * 0.1, V * 0.0, V * 0.2], 1.0)
        with pytest.raises(pstd.PstdError) as e:
            g.set_incidence_aux(0, KHAT, K, AXIS[0], AXIS[1], prof)
        assert e.value.code == "EINVAL"
