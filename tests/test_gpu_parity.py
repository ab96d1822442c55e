"""GPU parity: the CUDA path through the C ABI against the FP64 CPU oracle.

Tolerances (relative L2 unless stated), from the arithmetic:
  * FP64 path: 1e-12 after one step, 1e-10 after a full 750-step run (round-off of
    the two FFT orders growing along the run), transforms 1e-10 (the G = 8 cell
    quadrature reproduces the paper's sinc sum to ~1e-14 on these grids).
  * FP32 path: 2e-6 after one step, 2e-4 on psi after a full run and 1e-3 on
    cross-sections (single-precision round-off of ~6e-8 per operation over the
    FFT depth and the run).
"""
import dataclasses
import math

import numpy as np
import pytest

from oracle import analytic as an
from oracle import ntdf_oracle as no
from oracle import pstd_oracle as po
from paper_2403_04053_gb300 import inputs, pstd

pytestmark = pytest.mark.gpu

K = 2 * math.pi
E0 = 0.5 * K * K


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def ragged_spec(mode="exact"):
    # x spans one partial 32-lane tile, y one full tile, z two tiles with a ragged tail
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


# ----------------------------------------------------------------------------------
# one step from random states, several grid shapes
# ----------------------------------------------------------------------------------
ONE_STEP_SPECS = {
    "ragged-24x32x48": lambda mode: ragged_spec(mode),
    "cube-48": lambda mode: inputs.GridSpec(n=(48,) * 3, d=(0.25,) * 3, dt=0.004, tfsf_mode=mode),
    "mixed-96x16x64": lambda mode: inputs.GridSpec(n=(96, 16, 64), d=(0.2, 0.35, 0.25), dt=0.002, abc_cells=(8, 2, 6),
                                                   tfsf_lo=(30, 5, 20), tfsf_hi=(66, 11, 44), taper_cells=3,
                                                   huygens_lo=(20, 3, 12), huygens_hi=(76, 13, 52), tfsf_mode=mode),
    # square planes: the fused x+y pass (one CTA per z plane) on steps without the DFT
    "square-64x64x48": lambda mode: inputs.GridSpec(n=(64, 64, 48), d=(0.25, 0.25, 0.3), dt=0.002, abc_cells=(6, 6, 5),
                                                    tfsf_lo=(20, 20, 16), tfsf_hi=(44, 44, 32), taper_cells=3,
                                                    huygens_lo=(14, 14, 10), huygens_hi=(50, 50, 38), tfsf_mode=mode),
    "square-96x96x24": lambda mode: inputs.GridSpec(n=(96, 96, 24), d=(0.2, 0.2, 0.3), dt=0.001, abc_cells=(8, 8, 3),
                                                    tfsf_lo=(36, 36, 9), tfsf_hi=(60, 60, 15), taper_cells=2,
                                                    huygens_lo=(28, 28, 6), huygens_hi=(68, 68, 18), tfsf_mode=mode),
    # long y and z lines: the pipelined y pass (FP32, N = 192) and N = 256 z lines
    "pipe-16x192x256": lambda mode: inputs.GridSpec(n=(16, 192, 256), d=(0.3, 0.1, 0.08), dt=0.0005,
                                                    abc_cells=(2, 16, 20), tfsf_lo=(5, 60, 80), tfsf_hi=(11, 132, 176),
                                                    taper_cells=1, huygens_lo=(3, 40, 50), huygens_hi=(13, 150, 206),
                                                    tfsf_mode=mode),
    # 384-point lines (radix 12 x 8 x 4) along each axis in turn
    "line384-x": lambda mode: inputs.GridSpec(n=(384, 16, 12), d=(0.1, 0.3, 0.4), dt=0.0015, abc_cells=(24, 2, 1),
                                              tfsf_lo=(120, 5, 4), tfsf_hi=(264, 11, 8), taper_cells=1,
                                              huygens_lo=(100, 3, 2), huygens_hi=(284, 13, 10), tfsf_mode=mode),
    "line384-y": lambda mode: inputs.GridSpec(n=(16, 384, 12), d=(0.3, 0.1, 0.4), dt=0.0015, abc_cells=(2, 24, 1),
                                              tfsf_lo=(5, 120, 4), tfsf_hi=(11, 264, 8), taper_cells=1,
                                              huygens_lo=(3, 100, 2), huygens_hi=(13, 284, 10), tfsf_mode=mode),
    "line384-z": lambda mode: inputs.GridSpec(n=(12, 16, 384), d=(0.4, 0.3, 0.1), dt=0.0015, abc_cells=(1, 2, 24),
                                              tfsf_lo=(4, 5, 120), tfsf_hi=(8, 11, 264), taper_cells=1,
                                              huygens_lo=(2, 3, 100), huygens_hi=(10, 13, 284), tfsf_mode=mode),
    "radix3-12x192x8": lambda mode: inputs.GridSpec(n=(12, 192, 8), d=(0.3, 0.1, 0.4), dt=0.001, abc_cells=(2, 16, 1),
                                                    tfsf_lo=(4, 60, 3), tfsf_hi=(8, 132, 5), taper_cells=1,
                                                    huygens_lo=(3, 40, 2), huygens_hi=(9, 150, 6), tfsf_mode=mode),
    # 256-point x lines and 256-point y lines (radix 16 x 16; the y lines take the pipelined
    # pass in FP32 by default), the line lengths of the batched 256^3 configuration
    "line256-x": lambda mode: inputs.GridSpec(n=(256, 16, 12), d=(0.1, 0.3, 0.4), dt=0.0015, abc_cells=(20, 2, 1),
                                              tfsf_lo=(80, 5, 4), tfsf_hi=(176, 11, 8), taper_cells=1,
                                              huygens_lo=(60, 3, 2), huygens_hi=(196, 13, 10), tfsf_mode=mode),
    "line256-y": lambda mode: inputs.GridSpec(n=(16, 256, 12), d=(0.3, 0.1, 0.4), dt=0.0015, abc_cells=(2, 20, 1),
                                              tfsf_lo=(5, 80, 4), tfsf_hi=(11, 176, 8), taper_cells=1,
                                              huygens_lo=(3, 60, 2), huygens_hi=(13, 196, 10), tfsf_mode=mode),
    # square 192^2 and 256^2 planes: in FP32 the cluster-fused x+y pass (N / 32 CTAs a plane)
    "square-256x256x12": lambda mode: inputs.GridSpec(n=(256, 256, 12), d=(0.1, 0.1, 0.4), dt=0.0009,
                                                      abc_cells=(20, 20, 1), tfsf_lo=(80, 80, 4), tfsf_hi=(176, 176, 8),
                                                      taper_cells=1, huygens_lo=(60, 60, 2), huygens_hi=(196, 196, 10),
                                                      tfsf_mode=mode),
    "square-192x192x12": lambda mode: inputs.GridSpec(n=(192, 192, 12), d=(0.1, 0.12, 0.4), dt=0.001,
                                                      abc_cells=(16, 16, 1), tfsf_lo=(60, 60, 4), tfsf_hi=(132, 132, 8),
                                                      taper_cells=1, huygens_lo=(40, 40, 2), huygens_hi=(150, 150, 10),
                                                      tfsf_mode=mode),
    # 128^2 planes: the fused x+y pass as one CTA per plane or as a cluster of 4 CTAs
    "square-128x128x16": lambda mode: inputs.GridSpec(n=(128, 128, 16), d=(0.25, 0.2, 0.3), dt=0.002,
                                                      abc_cells=(10, 10, 2), tfsf_lo=(44, 44, 5), tfsf_hi=(84, 84, 11),
                                                      taper_cells=2, huygens_lo=(36, 36, 3), huygens_hi=(92, 92, 13),
                                                      tfsf_mode=mode),
    # z lines of 128, 192 and 256 points: the tensor-copy-fed z pass (FP32)
    "line256-z": lambda mode: inputs.GridSpec(n=(48, 12, 256), d=(0.3, 0.4, 0.1), dt=0.0015, abc_cells=(3, 1, 20),
                                              tfsf_lo=(12, 4, 80), tfsf_hi=(28, 8, 176), taper_cells=1,
                                              huygens_lo=(8, 2, 60), huygens_hi=(32, 10, 196), tfsf_mode=mode),
    "line128-z": lambda mode: inputs.GridSpec(n=(24, 16, 128), d=(0.3, 0.3, 0.15), dt=0.002, abc_cells=(2, 2, 10),
                                              tfsf_lo=(8, 5, 40), tfsf_hi=(16, 11, 88), taper_cells=1,
                                              huygens_lo=(5, 3, 30), huygens_hi=(19, 13, 98), tfsf_mode=mode),
    "line192-z": lambda mode: inputs.GridSpec(n=(32, 8, 192), d=(0.3, 0.4, 0.12), dt=0.002, abc_cells=(3, 1, 16),
                                              tfsf_lo=(9, 3, 60), tfsf_hi=(23, 5, 132), taper_cells=1,
                                              huygens_lo=(5, 2, 40), huygens_hi=(27, 6, 150), tfsf_mode=mode),
    # the paper's own absorber profile (Eq. Poshcl-Teller) on the ragged grid
    "ragged-poschl-teller": lambda mode: dataclasses.replace(ragged_spec(mode), abc_profile="poschl_teller",
                                                             abc_param=(5.0, 0.3)),
}


@pytest.mark.parametrize("prec,tol", [(pstd.F64, 1e-12), (pstd.F32, 2e-6)])
@pytest.mark.parametrize("mode", ["exact", "paper"])
@pytest.mark.parametrize("name", list(ONE_STEP_SPECS))
def test_one_step_matches_oracle(name, mode, prec, tol):
    spec = ONE_STEP_SPECS[name](mode)
    V = random_core_V(spec, 3)
    khat = (0.3, -0.5, 0.81)
    prev = inputs.random_field(spec.shape, 5)
    cur = inputs.random_field(spec.shape, 6)
    sim = po.Simulation(spec, V, khat, K, 0.05)
    sim.prev, sim.cur, sim.n = prev.copy(), cur.copy(), 17
    sim.step(1)
    cd = np.complex128 if prec == pstd.F64 else np.complex64
    with pstd.Grid(spec, precision=prec) as g:
        g.set_potential(V)
        g.set_incidence(0, khat, K, 0.05)
        g.set_field(0, prev.astype(cd), cur.astype(cd), 17)
        g.step(1)
        g.synchronize()
        assert g.get_step() == 18
        got = g.get_field(0)
        assert rel(got, sim.cur) < tol
        # the previous level is the old current one, untouched
        assert np.array_equal(g.get_field(0, pstd.FIELD_PREVIOUS), cur.astype(cd))


# ----------------------------------------------------------------------------------
# short runs with the running DFT, transforms and the far field
# ----------------------------------------------------------------------------------
@pytest.fixture(scope="module", params=["exact", "paper"])
def short_run(request):
    spec = ragged_spec(request.param)
    V = random_core_V(spec, 1)
    khat, w0 = (0.3, -0.5, 0.81), K * K / 2
    win = (20, 40)
    om = [w0, 0.93 * w0]
    sim = po.Simulation(spec, V, khat, K, 0.05, window=win, omegas=om)
    sim.step(60)
    pts = np.array([[3.0, -2.0, 5.5], [-4.0, 6.0, 1.0], [0.5, 0.2, -9.0], [30.0, 10.0, 40.0], [-200.0, 50.0, 120.0]])
    th = np.deg2rad(np.array([0.0, 33.0, 90.0, 140.0, 180.0]))
    ph = np.deg2rad(np.array([0.0, 20.0, 200.0, 300.0, 10.0]))
    # the transform of frequency f's phasors uses the free wavenumber at that energy, sqrt(2 w_f)
    ref = {f: (sim.scaled_phasors(f), no.transform_to_points(spec, math.sqrt(2 * om[f]), sim.scaled_phasors(f), pts),
               no.cross_section(spec, math.sqrt(2 * om[f]), sim.scaled_phasors(f), th, ph)) for f in range(2)}
    return dict(spec=spec, V=V, khat=khat, win=win, om=om, sim=sim, pts=pts, th=th, ph=ph, ref=ref)


@pytest.mark.parametrize("prec,tol_state,tol_out", [(pstd.F64, 1e-12, 1e-10), (pstd.F32, 2e-5, 2e-4)])
def test_short_run_dft_transform_far_field(short_run, prec, tol_state, tol_out):
    r = short_run
    with pstd.Grid(r["spec"], precision=prec) as g:
        g.set_potential(r["V"])
        g.set_incidence(0, r["khat"], K, 0.05)
        g.huygens_dft(0, r["om"], *r["win"])
        g.step(60)
        g.synchronize()
        assert rel(g.get_field(0), r["sim"].cur) < tol_state
        if r["spec"].tfsf_mode == "paper":
            assert rel(g.get_field(0, pstd.FIELD_SCATTERED), r["sim"].scattered_field()) < tol_state
        for f in range(2):
            phs, psi_ref, (ds_ref, f_ref) = r["ref"][f]
            for (gp, gd), (rp, rd) in zip(g.get_phasors(0, f), phs):
                assert rel(gp, rp) < 10 * tol_state and rel(gd, rd) < 10 * tol_state
            psi = g.transform_to_points(0, f, r["pts"])
            assert np.max(np.abs(psi - psi_ref) / np.abs(psi_ref)) < tol_out
            ds, fa = g.cross_section(0, f, r["th"], r["ph"])
            assert np.max(np.abs(fa - f_ref) / np.abs(f_ref)) < tol_out
            assert np.max(np.abs(ds - ds_ref) / ds_ref) < 2 * tol_out


def _runnable(spec, **kw):
    # a two-cell taper, so that the PAPER form's source (the taper's derivatives) is non-zero
    return dataclasses.replace(spec, taper_cells=2, **kw)


# (spec, steps, DFT window): Huygens planes close enough to the core that every face carries
# the scattered wave (at least 1% of the largest face's phasor norm) by the window's end
RUN_SPECS = {
    "ragged-poschl-teller": lambda mode: (ONE_STEP_SPECS["ragged-poschl-teller"](mode), 60, (20, 40)),
    "line256-x": lambda mode: (_runnable(ONE_STEP_SPECS["line256-x"](mode), huygens_lo=(72, 3, 2),
                                                   huygens_hi=(184, 13, 10)), 100, (40, 60)),
    "line256-y": lambda mode: (_runnable(ONE_STEP_SPECS["line256-y"](mode), huygens_lo=(3, 72, 2),
                                                   huygens_hi=(13, 184, 10)), 100, (40, 60)),
    "square-256x256x12": lambda mode: (_runnable(ONE_STEP_SPECS["square-256x256x12"](mode), huygens_lo=(72, 72, 2),
                                                 huygens_hi=(184, 184, 10)), 100, (40, 60)),
    "square-192x192x12": lambda mode: (_runnable(ONE_STEP_SPECS["square-192x192x12"](mode),
                                                 huygens_lo=(54, 54, 2), huygens_hi=(138, 138, 10)), 100, (40, 60)),
}


@pytest.mark.parametrize("prec,tol_state,tol_ph", [(pstd.F64, 1e-12, 1e-10), (pstd.F32, 2e-5, 2e-4)])
@pytest.mark.parametrize("mode", ["exact", "paper"])
@pytest.mark.parametrize("name", list(RUN_SPECS))
def test_windowed_run_matches_oracle(name, mode, prec, tol_state, tol_ph):
    # a run with the running DFT over its last steps: the state and the phasors of all six
    # planes (the DFT variants of the passes on these line lengths, and the mask profile)
    spec, steps, win = RUN_SPECS[name](mode)
    V = random_core_V(spec, 1)
    khat = (0.3, -0.5, 0.81)
    sim = po.Simulation(spec, V, khat, K, 0.05, window=win, omegas=[E0])
    sim.step(steps)
    with pstd.Grid(spec, precision=prec) as g:
        g.set_potential(V)
        g.set_incidence(0, khat, K, 0.05)
        g.huygens_dft(0, [E0], *win)
        g.step(steps)
        assert rel(g.get_field(0), sim.cur) < tol_state
        got = g.get_phasors(0, 0)
    ref = sim.scaled_phasors(0)
    peak = max(np.linalg.norm(p) for p, _ in ref)
    for (gp, gd), (rp, rd) in zip(got, ref):
        assert np.linalg.norm(rp) > 1e-2 * peak          # the plane carries the wave, not round-off
        assert rel(gp, rp) < tol_ph and rel(gd, rd) < tol_ph


@pytest.mark.parametrize("G,tol", [(4, 1e-3), (6, 1e-8), (8, 1e-10)])
def test_transform_quadrature_order(short_run, G, tol):
    # FP64, so that only the cell quadrature differs from the oracle's literal mode sum: G = 4
    # misses interpolant modes near the planes' Nyquist limit (a worst case of ~1e-4 a mode),
    # G = 8 (the FP64 default) is exact to round-off; the far field does not depend on G
    r = short_run
    with pstd.Grid(r["spec"], precision=pstd.F64) as g:
        g.set_potential(r["V"])
        g.set_incidence(0, r["khat"], K, 0.05)
        g.huygens_dft(0, r["om"], *r["win"])
        g.step(60)
        ref_psi = r["ref"][0][1]
        psi_default = g.transform_to_points(0, 0, r["pts"])
        g.set_transform_order(G)
        psi = g.transform_to_points(0, 0, r["pts"])
        assert rel(psi, ref_psi) < tol
        _, f = g.cross_section(0, 0, r["th"], r["ph"])
        assert rel(f, r["ref"][0][2][1]) < 1e-10
        # the adjoint transform follows the order (its transpose identity against the forward)
        y = np.random.default_rng(3).standard_normal(len(r["pts"])) + 0j
        x = g.join_phasors(g.transform_adjoint(0, 0, r["pts"], y))
        assert np.all(np.isfinite(x))
        g.set_transform_order(0)
        assert np.array_equal(g.transform_to_points(0, 0, r["pts"]), psi_default)
        with pytest.raises(pstd.PstdError) as e:
            g.set_transform_order(5)
        assert e.value.code == "EINVAL"


# ----------------------------------------------------------------------------------
# the full 48^3 square-barrier run (750 steps)
# ----------------------------------------------------------------------------------
@pytest.fixture(scope="module")
def barrier_run():
    wl = inputs.square_barrier_workload()
    inc = wl.incidences[0]
    sim = po.Simulation(wl.spec, wl.V, inc.khat, inc.k, inc.ramp_time, window=(wl.window_first, wl.window_len))
    sim.step(wl.nsteps)
    phs = sim.scaled_phasors(0)
    ds, f = no.cross_section(wl.spec, K, phs, wl.far_theta, wl.far_phi)
    sub = wl.fresnel_points[::97]
    psi = no.transform_to_points(wl.spec, K, phs, sub)
    return wl, sim, ds, f, sub, psi


def _run_gpu(wl, prec):
    g = pstd.Grid(wl.spec, precision=prec)
    pstd.setup_workload(g, wl)
    g.step(wl.nsteps)
    g.synchronize()
    return g


def test_square_barrier_full_run_fp64(barrier_run):
    wl, sim, ds_ref, f_ref, sub, psi_ref = barrier_run
    with _run_gpu(wl, pstd.F64) as g:
        assert rel(g.get_field(0), sim.cur) < 1e-10
        ds, f = g.cross_section(0, 0, wl.far_theta, wl.far_phi)
        assert rel(f, f_ref) < 1e-10
        assert rel(g.transform_to_points(0, 0, sub), psi_ref) < 1e-10
        # and the physics: within 3% of the analytic partial waves (voxelised sphere)
        pw = np.abs(an.partial_wave_amplitude(wl.far_theta, K, 0.3 * E0, 1.5)) ** 2
        assert rel(ds, pw) < 3e-2
        # the full 32 x 32 Fresnel plane at z = 20 runs and is finite
        full = g.transform_to_points(0, 0, wl.fresnel_points)
        assert full.shape == (1024,) and np.all(np.isfinite(full))


def test_square_barrier_converges_to_partial_waves_under_refinement():
    """The same sphere (V0 = 0.3 E0, a = 1.5) at half the spacing: dx = 0.125 (96^3, 12 cells a
    radius), dt / 4, 3000 steps over the same physical times, FP64.  The 48^3 run's 2.2% miss is
    the volume-fraction voxelisation of the sphere at six cells a radius: halving dx takes the
    error under the 1% target (relative L2 of dsigma/dOmega over 181 angles)."""
    errs = []
    pw = None
    for f in (1, 2):
        wl = inputs.square_barrier_workload(n=48 * f, dx=0.25 / f, dt=0.004 / f / f, nsteps=750 * f * f,
                                            ramp_steps=125 * f * f, abc=8 * f, tf=(14 * f, 34 * f), taper=4 * f,
                                            hb=(11 * f, 37 * f))
        with _run_gpu(wl, pstd.F64) as g:
            ds, _ = g.cross_section(0, 0, wl.far_theta, wl.far_phi)
        pw = np.abs(an.partial_wave_amplitude(wl.far_theta, K, 0.3 * E0, 1.5)) ** 2
        errs.append(rel(ds, pw))
    assert errs[0] < 3e-2 and errs[1] < 1e-2 and errs[1] < 0.5 * errs[0], errs


def test_square_barrier_full_run_fp32_against_fp64_oracle(barrier_run):
    wl, sim, ds_ref, f_ref, sub, psi_ref = barrier_run
    with _run_gpu(wl, pstd.F32) as g:
        assert rel(g.get_field(0), sim.cur) < 2e-4
        ds, f = g.cross_section(0, 0, wl.far_theta, wl.far_phi)
        assert rel(ds, ds_ref) < 1e-3
        assert rel(g.transform_to_points(0, 0, sub), psi_ref) < 1e-3


# ----------------------------------------------------------------------------------
# the 128^3 Gaussian-sum geometry, in the launch configuration the benchmark times
# ----------------------------------------------------------------------------------
@pytest.fixture(scope="module")
def big():
    wl = inputs.gaussian_sum_workload(with_outputs=False)
    return wl


@pytest.mark.parametrize("prec,tol", [(pstd.F64, 1e-12), (pstd.F32, 2e-6)])
def test_128_cubed_one_step_elementwise(big, prec, tol):
    wl = big
    inc = wl.incidences[0]
    prev = inputs.smooth_random_field(wl.spec, 7)
    cur = inputs.smooth_random_field(wl.spec, 8)
    sim = po.Simulation(wl.spec, wl.V, inc.khat, inc.k, inc.ramp_time)
    sim.prev, sim.cur, sim.n = prev.copy(), cur.copy(), 200
    sim.step(1)
    cd = np.complex128 if prec == pstd.F64 else np.complex64
    with pstd.Grid(wl.spec, precision=prec) as g:
        g.set_potential(wl.V)
        g.set_incidence(0, inc.khat, inc.k, inc.ramp_time)
        g.set_field(0, prev.astype(cd), cur.astype(cd), 200)
        g.step(1)
        got = g.get_field(0)
    assert rel(got, sim.cur) < tol
    assert np.max(np.abs(got - sim.cur)) < 20 * tol * np.max(np.abs(sim.cur))


def plane128_spec():
    """128 x 128 planes (the fused x+y pass with its plane DFT in FP32), 32 z planes: a smooth
    scatterer in the core whose wave reaches all six Huygens planes well before the window ends."""
    return inputs.GridSpec(n=(128, 128, 32), d=(0.25, 0.25, 0.25), dt=0.0036, abc_cells=(12, 12, 4), tfsf_lo=(44, 44, 9),
                           tfsf_hi=(84, 84, 23), taper_cells=3, huygens_lo=(36, 36, 6), huygens_hi=(92, 92, 26))


def plane128_V(spec):
    # seeded random values on an 8 x 8 x 6 block at the centre: a rough scatterer that sends
    # its wave in every direction, so that the back faces carry more than round-off
    rng = np.random.default_rng(128)
    V = np.zeros(spec.shape)
    V[13:19, 60:68, 60:68] = rng.uniform(-0.4 * E0, 0.4 * E0, (6, 8, 8))
    return V


PLANE128_WINDOW = (250, 150)


@pytest.fixture(scope="module")
def plane128_run():
    spec = plane128_spec()
    V = plane128_V(spec)
    sim = po.Simulation(spec, V, (0.3, -0.5, 0.81), K, 0.3, window=PLANE128_WINDOW, omegas=[E0])
    sim.step(sum(PLANE128_WINDOW))
    return spec, V, sim


@pytest.mark.parametrize("prec,tol_state,tol_ph", [(pstd.F64, 1e-11, 1e-10), (pstd.F32, 2e-5, 2e-5)])
def test_128_planes_windowed_run_phasors_elementwise(plane128_run, prec, tol_state, tol_ph):
    # 400 steps, the last 150 in the DFT window: in FP32 every step runs the fused x+y pass on
    # the 128^2 planes (with the x- and y-plane DFT on window steps); the scattered wave has
    # reached every Huygens plane, so each face's phasors are compared by relative L2 on their
    # own scale (their norm is checked to be far above round-off)
    spec, V, sim = plane128_run
    with pstd.Grid(spec, precision=prec) as g:
        g.set_potential(V)
        g.set_incidence(0, (0.3, -0.5, 0.81), K, 0.3)
        g.huygens_dft(0, [E0], *PLANE128_WINDOW)
        g.set_timing(True)
        g.step(sum(PLANE128_WINDOW))
        if prec == pstd.F32:
            assert g.kernel_stats("xypass")[0] == sum(PLANE128_WINDOW)
        assert rel(g.get_field(0), sim.cur) < tol_state
        got = g.get_phasors(0, 0)
    ref = sim.scaled_phasors(0)
    peak = max(np.max(np.abs(p)) for p, _ in ref)
    for (gp, gd), (rp, rd) in zip(got, ref):
        assert np.max(np.abs(rp)) > 1e-3 * peak       # each plane carries the wave, not round-off
        assert rel(gp, rp) < tol_ph and rel(gd, rd) < tol_ph


@pytest.mark.parametrize("prec,tol", [(pstd.F64, 1e-10), (pstd.F32, 1e-4)])
def test_128_cubed_sampled_transform(big, prec, tol):
    """Phasors from a short 128^3 run; the surface transform at sampled Fresnel-plane points and
    far-field directions against the oracle's literal mode sum on the GPU's own phasors."""
    wl = big
    inc = wl.incidences[0]
    w0 = K * K / 2
    with pstd.Grid(wl.spec, precision=prec) as g:
        g.set_potential(wl.V)
        g.set_incidence(0, inc.khat, inc.k, 0.05)
        g.huygens_dft(0, [w0], 20, 30)
        g.step(50)
        phs = g.get_phasors(0, 0)
        D = 18.0
        pts = inputs.plane_points(inc.khat, D * D / 4, 1.5 * D, 256)[[0, 33000, 65535]]
        psi = g.transform_to_points(0, 0, pts)
        th = np.deg2rad([5.0, 91.0, 170.0])
        ph = np.deg2rad([10.0, 250.0, 0.0])
        ds, f = g.cross_section(0, 0, th, ph)
    ref = no.transform_to_points(wl.spec, K, phs, pts)
    _, fref = no.cross_section(wl.spec, K, phs, th, ph)
    assert np.max(np.abs(psi - ref) / np.abs(ref)) < tol
    assert np.max(np.abs(f - fref) / np.abs(fref)) < tol


# ----------------------------------------------------------------------------------
# edge cases and ABI behaviour
# ----------------------------------------------------------------------------------
def test_exact_form_leaks_nothing_at_zero_potential():
    wl = inputs.square_barrier_workload(with_outputs=False)
    for prec in (pstd.F32, pstd.F64):
        with pstd.Grid(wl.spec, precision=prec) as g:
            g.set_potential(np.zeros(wl.spec.shape))
            g.set_incidence(0, (0.36, 0.48, 0.8), K, 0.5)
            g.step(300)
            assert np.count_nonzero(g.get_field(0)) == 0


def test_batched_members_equal_separate_runs():
    spec = ragged_spec()
    V = random_core_V(spec, 2)
    dirs = [(0.3, -0.5, 0.81), (-0.6, 0.0, 0.8)]
    w0 = K * K / 2
    outs = []
    for b, kh in enumerate(dirs):
        with pstd.Grid(spec, precision=pstd.F32) as g:
            g.set_potential(V)
            g.set_incidence(0, kh, K, 0.05)
            g.huygens_dft(0, [w0], 10, 20)
            g.step(30)
            outs.append((g.get_field(0), g.transform_to_points(0, 0, [[5.0, 5.0, 9.0]])))
    with pstd.Grid(spec, precision=pstd.F32, batch=2) as g:
        g.set_potential(V)
        for b, kh in enumerate(dirs):
            g.set_incidence(b, kh, K, 0.05)
        g.huygens_dft(-1, [w0], 10, 20)
        g.step(30)
        for b in range(2):
            assert np.array_equal(g.get_field(b), outs[b][0])
            assert np.array_equal(g.transform_to_points(b, 0, [[5.0, 5.0, 9.0]]), outs[b][1])


@pytest.mark.parametrize("prec,tol", [(pstd.F64, 1e-12), (pstd.F32, 1e-5)])
def test_transform_members_equals_single_member_transforms(prec, tol):
    # three members, two wavenumbers, two DFT frequencies, in one launch: each row must be the
    # single-member transform of that member and frequency
    spec = ragged_spec()
    V = random_core_V(spec, 2)
    incs = [((0.3, -0.5, 0.81), K), ((-0.6, 0.0, 0.8), K), ((0.0, 0.6, 0.8), K / 2)]
    pts = np.array([[3.0, -2.0, 5.5], [30.0, 10.0, 40.0], [-200.0, 50.0, 120.0], [0.5, 0.2, -9.0]])
    with pstd.Grid(spec, precision=prec, batch=3) as g:
        g.set_potential(V)
        for b, (kh, k) in enumerate(incs):
            g.set_incidence(b, kh, k, 0.05)
            g.huygens_dft(b, [0.5 * k * k, 0.45 * k * k], 10, 20)
        g.step(30)
        order, freqs = [0, 2, 1, 0], [0, 1, 0, 1]
        got = g.transform_members(order, freqs, pts)
        for row, (b, f) in enumerate(zip(order, freqs)):
            assert rel(got[row], g.transform_to_points(b, f, pts)) < tol
        import torch
        dev = g.transform_members(order, freqs, torch.from_numpy(pts).cuda()).cpu().numpy()
        assert np.array_equal(dev, got)


def test_batched_256_cube_shell_transform_against_the_oracle():
    # the batched configuration at full size (16 incidences, 256^3, FP32): all sixteen members
    # transformed in one call to seeded points of the shell 0.5 D^2/lambda .. 4 D^2/lambda; the
    # members with k = 2 pi and k = pi checked at two points against the oracle's literal mode
    # sum of the GPU's own phasors, and every member against its single-member transform
    from oracle import ntdf_oracle as no_
    wl = inputs.batched_workload()
    spec = wl.spec
    B = len(wl.incidences)
    D = (spec.tfsf_hi[0] - spec.taper_cells - (spec.tfsf_lo[0] + spec.taper_cells)) * spec.d[0]
    pts = inputs.shell_points(64, 0.5 * D * D, 4.0 * D * D, 2408)
    with pstd.Grid(spec, precision=pstd.F32, batch=B) as g:
        g.set_potential(wl.V)
        for b, inc in enumerate(wl.incidences):
            g.set_incidence(b, inc.khat, inc.k, inc.ramp_time)
            g.huygens_dft(b, [0.5 * inc.k ** 2], 700, 200)
        g.step(900)            # the scattered waves have reached the Huygens planes
        got = g.transform_members(list(range(B)), [0] * B, pts)
        for b in (0, 5, 9, 15):
            assert rel(got[b], g.transform_to_points(b, 0, pts)) < 1e-5
        for b in (3, 12):
            k = wl.incidences[b].k
            ref = no_.transform_to_points(spec, k, g.get_phasors(b, 0), pts[[7, 23, 40]])
            assert rel(got[b][[7, 23, 40]], ref) < 1e-4


def test_device_buffers_match_host_buffers():
    import torch
    spec = ragged_spec()
    V = random_core_V(spec, 4)
    w0 = K * K / 2
    pts = np.array([[3.0, -2.0, 5.5], [30.0, 10.0, 40.0]])
    th, ph = np.deg2rad([10.0, 100.0]), np.deg2rad([5.0, 60.0])
    with pstd.Grid(spec, precision=pstd.F64) as g:
        g.set_potential(torch.from_numpy(V).cuda())
        g.set_incidence(0, (0, 0, 1), K, 0.05)
        g.huygens_dft(0, [w0], 10, 20)
        g.step(30)
        a = g.transform_to_points(0, 0, pts)
        b = g.transform_to_points(0, 0, torch.from_numpy(pts).cuda()).cpu().numpy()
        assert np.array_equal(a, b)
        ds, f = g.cross_section(0, 0, th, ph)
        ds2, f2 = g.cross_section(0, 0, torch.from_numpy(th).cuda(), torch.from_numpy(ph).cuda())
        assert np.array_equal(f, f2.cpu().numpy()) and np.array_equal(ds, ds2.cpu().numpy())
        out = torch.empty(spec.shape, dtype=torch.complex128, device="cuda")
        g.get_field(0, out=out)
        assert np.array_equal(out.cpu().numpy(), g.get_field(0))


def test_runs_are_bitwise_deterministic():
    spec = ragged_spec()
    V = random_core_V(spec, 5)
    res = []
    for _ in range(2):
        with pstd.Grid(spec, precision=pstd.F32) as g:
            g.set_potential(V)
            g.set_incidence(0, (0.3, -0.5, 0.81), K, 0.05)
            g.huygens_dft(0, [K * K / 2], 10, 20)
            g.step(30)
            res.append((g.get_field(0), g.cross_section(0, 0, [0.3], [0.2])[1]))
    assert np.array_equal(res[0][0], res[1][0]) and np.array_equal(res[0][1], res[1][1])


def test_nonfinite_state_is_reported():
    spec = ragged_spec()
    with pstd.Grid(spec, precision=pstd.F32) as g:
        g.set_incidence(0, (0, 0, 1), K, 0.05)
        bad = np.zeros(spec.shape, dtype=np.complex64)
        bad[10, 10, 10] = np.nan
        g.set_field(0, bad, bad, 0)
        g.step(1)
        with pytest.raises(pstd.PstdError) as e:
            g.synchronize()
        assert e.value.code == "ENONFINITE"
        g.synchronize()   # the flag is cleared once reported


def test_call_order_errors():
    spec = ragged_spec()
    with pstd.Grid(spec, precision=pstd.F32) as g:
        with pytest.raises(pstd.PstdError) as e:
            g.step(1)
        assert e.value.code == "ESTATE"
        g.set_incidence(0, (0, 0, 1), K, 0.05)
        g.huygens_dft(0, [K * K / 2], 5, 10)
        g.step(8)
        with pytest.raises(pstd.PstdError) as e:
            g.transform_to_points(0, 0, [[5.0, 5.0, 5.0]])
        assert e.value.code == "ESTATE"
        with pytest.raises(pstd.PstdError) as e:
            g.set_potential(np.ones(spec.shape))
        assert e.value.code == "EINVAL"
        with pytest.raises(pstd.PstdError) as e:
            g.cross_section(0, 3, [0.1], [0.1])
        assert e.value.code == "EINVAL"


def test_fused_xy_pass_with_and_without_the_dft():
    # 64^2 planes in FP32: the fused x+y pass runs on every step, with the x- and y-plane DFT
    # on the window steps, and the z pass carries the V-term and source throughout
    spec = ONE_STEP_SPECS["square-64x64x48"]("exact")
    V = random_core_V(spec, 4)
    khat, win = (0.3, -0.5, 0.81), (10, 10)
    sim = po.Simulation(spec, V, khat, K, 0.05, window=win, omegas=[E0, 0.9 * E0])
    sim.step(30)
    with pstd.Grid(spec, precision=pstd.F32) as g:
        g.set_potential(V)
        g.set_incidence(0, khat, K, 0.05)
        g.huygens_dft(0, [E0, 0.9 * E0], *win)
        g.set_timing(True)
        g.step(30)
        assert g.kernel_stats("xypass")[0] == 30
        assert g.kernel_stats("xpass")[0] == 0 and g.kernel_stats("ypass")[0] == 0
        assert g.kernel_stats("zpass")[0] == 30 and g.kernel_stats("source")[0] == 0
        assert rel(g.get_field(0), sim.cur) < 2e-5
        for f in range(2):
            ph, ref = g.get_phasors(0, f), sim.scaled_phasors(f)
            for a, b in zip(ph, ref):
                assert rel(a[0], b[0]) < 2e-5 and rel(a[1], b[1]) < 2e-5


def test_timing_and_launch_counts():
    spec = ragged_spec()
    with pstd.Grid(spec, precision=pstd.F32) as g:
        g.set_incidence(0, (0, 0, 1), K, 0.05)
        g.set_timing(True)
        g.step(5)
        for name in ("xpass", "ypass", "zpass"):
            n, ms = g.kernel_stats(name)
            assert n == 5 and ms > 0
        assert g.launch_count() == 15


def test_batched_256_cube_matches_separate_runs():
    # the batched configuration at full size: 16 incidences on one potential (256^3, FP32),
    # 12 steps with every member's DFT window over steps 4..11; members 3 and 12 (k = 2 pi and
    # k = pi) stepped in a batch of two with member 0 (whose energy sets the absorber) give the
    # same state and phasors
    wl = inputs.batched_workload()
    spec = wl.spec
    B = len(wl.incidences)

    def setup(g, members):
        g.set_potential(wl.V)
        for b, i in enumerate(members):
            inc = wl.incidences[i]
            g.set_incidence(b, inc.khat, inc.k, inc.ramp_time)
            g.huygens_dft(b, [0.5 * inc.k ** 2], 4, 8)

    with pstd.Grid(spec, precision=pstd.F32, batch=B) as g:
        setup(g, range(B))
        g.step(12)
        got = {i: (g.get_field(i), g.get_phasors(i, 0)) for i in (3, 12)}
    for i in (3, 12):
        with pstd.Grid(spec, precision=pstd.F32, batch=2) as g1:
            setup(g1, [0, i])
            g1.step(12)
            assert rel(got[i][0], g1.get_field(1)) < 1e-6
            for a, b in zip(got[i][1], g1.get_phasors(1, 0)):
                assert rel(a[0], b[0]) < 1e-6 and rel(a[1], b[1]) < 1e-6


# ----------------------------------------------------------------------------------
# Gaussian wave-packet incidence and many DFT frequencies
# ----------------------------------------------------------------------------------
PACKET = (0.6, -1.0)   # sigma, d0: the packet overlaps the scatterer within a few steps


@pytest.mark.parametrize("prec,tol", [(pstd.F64, 1e-12), (pstd.F32, 2e-6)])
def test_packet_one_step_matches_oracle(prec, tol):
    spec = ragged_spec("exact")
    V = random_core_V(spec, 3)
    khat = (0.3, -0.5, 0.81)
    prev = inputs.random_field(spec.shape, 5)
    cur = inputs.random_field(spec.shape, 6)
    sim = po.Simulation(spec, V, khat, K, 0.0, packet=PACKET)
    sim.prev, sim.cur, sim.n = prev.copy(), cur.copy(), 17
    sim.step(1)
    cd = np.complex128 if prec == pstd.F64 else np.complex64
    with pstd.Grid(spec, precision=prec) as g:
        g.set_potential(V)
        g.set_incidence_packet(0, khat, K, *PACKET)
        g.set_field(0, prev.astype(cd), cur.astype(cd), 17)
        g.step(1)
        assert rel(g.get_field(0), sim.cur) < tol


@pytest.mark.parametrize("prec,tol_state,tol_out", [(pstd.F64, 1e-12, 1e-10), (pstd.F32, 2e-5, 2e-4)])
def test_packet_run_with_many_frequencies(prec, tol_state, tol_out):
    # 60 steps, a 40-step window, 9 DFT frequencies across the packet's spectrum
    spec = ragged_spec("exact")
    V = random_core_V(spec, 1)
    khat = (0.3, -0.5, 0.81)
    om = list(np.linspace(0.8, 1.2, 9) * E0)
    sim = po.Simulation(spec, V, khat, K, 0.0, window=(20, 40), omegas=om, packet=PACKET)
    sim.step(60)
    pts = np.array([[3.0, -2.0, 5.5], [-4.0, 6.0, 1.0], [30.0, 10.0, 40.0]])
    with pstd.Grid(spec, precision=prec) as g:
        g.set_potential(V)
        g.set_incidence_packet(0, khat, K, *PACKET)
        g.huygens_dft(0, om, 20, 40)
        g.step(60)
        assert rel(g.get_field(0), sim.cur) < tol_state
        for f in (0, 4, 8):
            ref = sim.scaled_phasors(f)
            got = g.get_phasors(0, f)
            for a, b in zip(got, ref):
                assert rel(a[0], b[0]) < tol_out and rel(a[1], b[1]) < tol_out
            kf = math.sqrt(2 * om[f])
            assert rel(g.transform_to_points(0, f, pts), no.transform_to_points(spec, kf, ref, pts)) < tol_out


@pytest.mark.parametrize("prec", [pstd.F64, pstd.F32])
def test_packet_run_reproduces_cw_cross_sections(prec):
    # one packet run gives, at each DFT frequency, the scattering of a CW wave of that energy
    spec = inputs.GridSpec(n=(24, 24, 24), d=(0.25, 0.25, 0.25), dt=0.004, abc_cells=(4, 4, 4), tfsf_lo=(6, 6, 6),
                           tfsf_hi=(17, 17, 17), taper_cells=2, huygens_lo=(5, 5, 5), huygens_hi=(18, 18, 18))
    x = [spec.coords(a) for a in range(3)]
    Z, Y, X = np.meshgrid(x[2], x[1], x[0], indexing="ij")
    V = 6.0 * np.exp(-(X ** 2 + Y ** 2 + Z ** 2) / (2 * 0.5 ** 2))
    c = spec.core_box()
    inside = np.zeros(spec.shape, bool)
    inside[c[2][0]:c[2][1] + 1, c[1][0]:c[1][1] + 1, c[0][0]:c[0][1] + 1] = True
    V[~inside] = 0
    oms = [0.9 * E0, E0, 1.1 * E0]
    th, ph = np.deg2rad([10.0, 60.0, 120.0, 170.0]), np.zeros(4)
    with pstd.Grid(spec, precision=prec) as g:
        g.set_potential(V)
        g.set_incidence_packet(0, (0, 0, 1), K, 1.0, -6.0)
        g.huygens_dft(0, oms, 0, 1200)
        g.step(1200)
        fp = [g.cross_section(0, i, th, ph)[1] for i in range(3)]
    for i, (w, tol) in enumerate(zip(oms, (2e-2, 1e-3, 2e-2))):
        kw = math.sqrt(2 * w)
        with pstd.Grid(spec, precision=prec) as g:
            g.set_potential(V)
            g.set_incidence(0, (0, 0, 1), kw, 0.5)
            g.huygens_dft(0, [w], *inputs.dft_window(w, spec.dt, 900))
            g.step(900)
            fc = g.cross_section(0, 0, th, ph)[1]
        assert rel(fp[i], fc) < tol


def test_packet_call_errors():
    with pstd.Grid(ragged_spec("paper"), precision=pstd.F32) as g:
        with pytest.raises(pstd.PstdError) as e:
            g.set_incidence_packet(0, (0, 0, 1), K, 1.0, -2.0)
        assert e.value.code == "EINVAL"        # the packet needs the EXACT form
    with pstd.Grid(ragged_spec("exact"), precision=pstd.F32) as g:
        for sig in (0.0, -1.0):
            with pytest.raises(pstd.PstdError) as e:
                g.set_incidence_packet(0, (0, 0, 1), K, sig, -2.0)
            assert e.value.code == "EINVAL"
        with pytest.raises(pstd.PstdError) as e:
            g.huygens_dft(0, [E0] * (pstd.MAX_FREQ + 1), 0, 10)
        assert e.value.code == "EINVAL"
        g.set_incidence_packet(0, (0, 0, 1), K, 1.0, -2.0)
        g.huygens_dft(0, [E0] * pstd.MAX_FREQ, 0, 10)
        with pytest.raises(pstd.PstdError) as e:
            g.adjoint_gradient(10, [np.zeros(g.phasor_count() * pstd.MAX_FREQ)], (0, 0, 0), (4, 4, 4))
        assert e.value.code == "EINVAL"        # the adjoint supports the CW incidence


# ----------------------------------------------------------------------------------
# CUDA-graph replay of repeated runs
# ----------------------------------------------------------------------------------
def _windowed_runs(spec, V, graphs, passes, V_after=None):
    out = []
    with pstd.Grid(spec, precision=pstd.F32) as g:
        g.set_graphs(graphs)
        g.set_potential(V)
        g.set_incidence(0, (0.3, -0.5, 0.81), K, 0.05)
        g.huygens_dft(0, [E0], 10, 10)
        for p in range(passes):
            if V_after is not None and p == passes - 1:
                g.set_potential(V_after)
            g.reset()
            g.step(30)
            out.append((g.get_field(0), g.join_phasors(g.get_phasors(0, 0)), g.launch_count()))
        out.append(g.graph_replays())
    return out


def test_graph_replay_matches_direct_launches():
    # pass 1 launches directly, pass 2 is captured, pass 3 replays the graph
    spec = ONE_STEP_SPECS["square-64x64x48"]("exact")
    V = random_core_V(spec, 4)
    direct = _windowed_runs(spec, V, False, 3)
    graphed = _windowed_runs(spec, V, True, 3)
    assert direct[-1] == 0 and graphed[-1] == 2        # passes 2 and 3 ran as graph launches
    for (s0, p0, _), (s1, p1, _) in zip(direct[:-1], graphed[:-1]):
        assert np.array_equal(s0, s1) and np.array_equal(p0, p1)
    # the replayed passes count the same kernel launches as the direct ones
    assert [n for _, _, n in direct[:-1]] == [n for _, _, n in graphed[:-1]]


def test_graph_is_not_replayed_after_a_new_potential():
    spec = ONE_STEP_SPECS["square-64x64x48"]("exact")
    V1, V2 = random_core_V(spec, 4), random_core_V(spec, 5)
    graphed = _windowed_runs(spec, V1, True, 3, V_after=V2)
    fresh = _windowed_runs(spec, V2, False, 1)
    assert graphed[-1] == 1                            # only pass 2 replayed; pass 3 had a new V
    assert np.array_equal(graphed[-2][0], fresh[0][0]) and np.array_equal(graphed[-2][1], fresh[0][1])


# ----------------------------------------------------------------------------------
# step-kernel variants and the autotuner
# ----------------------------------------------------------------------------------
X, L = pstd, pstd
VARIANTS = [("square-64x64x48", (X.XY_PLANE, L.LINE_PLAIN, L.LINE_PLAIN)),
            ("square-64x64x48", (X.XY_SEPARATE, L.LINE_PLAIN, L.LINE_PLAIN)),
            ("pipe-16x192x256", (X.XY_SEPARATE, L.LINE_PIPELINED, L.LINE_PLAIN)),
            ("pipe-16x192x256", (X.XY_SEPARATE, L.LINE_TMA, L.LINE_TMA)),
            ("pipe-16x192x256", (X.XY_SEPARATE, L.LINE_PLAIN, L.LINE_PLAIN)),
            ("line256-y", (X.XY_SEPARATE, L.LINE_PIPELINED, L.LINE_PLAIN)),
            ("line256-y", (X.XY_SEPARATE, L.LINE_TMA, L.LINE_PLAIN)),
            ("line256-y", (X.XY_SEPARATE, L.LINE_PLAIN, L.LINE_PLAIN)),
            ("square-256x256x12", (X.XY_CLUSTER, L.LINE_PLAIN, L.LINE_PLAIN)),
            ("square-256x256x12", (X.XY_SEPARATE, L.LINE_PIPELINED, L.LINE_PLAIN)),
            ("square-256x256x12", (X.XY_SEPARATE, L.LINE_TMA, L.LINE_PLAIN)),
            ("square-256x256x12", (X.XY_SEPARATE, L.LINE_PLAIN, L.LINE_PLAIN)),
            ("square-192x192x12", (X.XY_CLUSTER, L.LINE_PLAIN, L.LINE_PLAIN)),
            ("square-128x128x16", (X.XY_PLANE, L.LINE_PLAIN, L.LINE_PLAIN)),
            ("square-128x128x16", (X.XY_CLUSTER, L.LINE_PLAIN, L.LINE_PLAIN)),
            ("square-128x128x16", (X.XY_SEPARATE, L.LINE_TMA, L.LINE_PLAIN)),
            ("line256-z", (X.XY_SEPARATE, L.LINE_PLAIN, L.LINE_TMA)),
            ("line256-z", (X.XY_SEPARATE, L.LINE_PLAIN, L.LINE_PLAIN)),
            ("line128-z", (X.XY_SEPARATE, L.LINE_PLAIN, L.LINE_TMA)),
            ("line192-z", (X.XY_SEPARATE, L.LINE_PLAIN, L.LINE_TMA)),
            # the alternative FFT plans (radix 8-8-4 at 256 points, 8-4-4 at 128)
            ("line256-x", (X.XY_SEPARATE, L.LINE_PLAIN, L.LINE_PLAIN, 0b001)),
            ("line256-y", (X.XY_SEPARATE, L.LINE_PLAIN, L.LINE_PLAIN, 0b010)),
            ("line256-z", (X.XY_SEPARATE, L.LINE_PLAIN, L.LINE_PLAIN, 0b100)),
            ("line128-z", (X.XY_SEPARATE, L.LINE_PLAIN, L.LINE_PLAIN, 0b100)),
            ("square-256x256x12", (X.XY_CLUSTER, L.LINE_PLAIN, L.LINE_PLAIN, 0b011)),
            ("square-256x256x12", (X.XY_SEPARATE, L.LINE_PLAIN, L.LINE_PLAIN, 0b011)),
            ("square-128x128x16", (X.XY_CLUSTER, L.LINE_PLAIN, L.LINE_PLAIN, 0b011)),
            ("square-128x128x16", (X.XY_SEPARATE, L.LINE_PLAIN, L.LINE_PLAIN, 0b011))]


@pytest.mark.parametrize("name,variants", VARIANTS)
def test_every_variant_matches_oracle(name, variants):
    spec = ONE_STEP_SPECS[name]("exact")
    V = random_core_V(spec, 3)
    khat = (0.3, -0.5, 0.81)
    prev = inputs.random_field(spec.shape, 5)
    cur = inputs.random_field(spec.shape, 6)
    sim = po.Simulation(spec, V, khat, K, 0.05)
    sim.prev, sim.cur, sim.n = prev.copy(), cur.copy(), 17
    sim.step(1)
    with pstd.Grid(spec, precision=pstd.F32) as g:
        g.set_variants(*variants)
        g.set_potential(V)
        g.set_incidence(0, khat, K, 0.05)
        g.set_field(0, prev.astype(np.complex64), cur.astype(np.complex64), 17)
        g.step(1)
        assert rel(g.get_field(0), sim.cur) < 2e-6


@pytest.mark.parametrize("name,variants", [("square-256x256x12", (pstd.XY_CLUSTER, 0, 0, 0b011)),
                                           ("square-256x256x12", (pstd.XY_SEPARATE, 0, 0, 0b011)),
                                           ("square-192x192x12", (pstd.XY_SEPARATE, 0, 0, 0))])
@pytest.mark.parametrize("prec", [pstd.F32])
def test_windowed_run_of_each_variant(name, variants, prec):
    # the DFT-window forms of the alternative-plan passes (cluster and separate) and of the
    # separate passes on 192-point lines
    spec, steps, win = RUN_SPECS[name]("exact")
    V = random_core_V(spec, 1)
    khat = (0.3, -0.5, 0.81)
    sim = po.Simulation(spec, V, khat, K, 0.05, window=win, omegas=[E0])
    sim.step(steps)
    with pstd.Grid(spec, precision=prec) as g:
        g.set_variants(*variants)
        g.set_potential(V)
        g.set_incidence(0, khat, K, 0.05)
        g.huygens_dft(0, [E0], *win)
        g.step(steps)
        assert rel(g.get_field(0), sim.cur) < 2e-5
        got = g.get_phasors(0, 0)
    for (gp, gd), (rp, rd) in zip(got, sim.scaled_phasors(0)):
        assert rel(gp, rp) < 2e-4 and rel(gd, rd) < 2e-4


def test_autotune_keeps_the_state_and_picks_available_variants():
    spec = ONE_STEP_SPECS["square-64x64x48"]("exact")
    V = random_core_V(spec, 3)
    with pstd.Grid(spec, precision=pstd.F32) as g:
        g.set_potential(V)
        g.set_incidence(0, (0.3, -0.5, 0.81), K, 0.05)
        g.step(7)
        before, n = g.get_field(0), g.get_step()
        chosen = g.autotune(10)
        assert chosen["y_pass"] == pstd.LINE_PLAIN      # 64-point y lines: only the plain y pass
        assert chosen["fused_xy"] in (pstd.XY_SEPARATE, pstd.XY_PLANE)
        assert g.get_step() == n and np.array_equal(g.get_field(0), before)
        for bad in ((pstd.XY_SEPARATE, pstd.LINE_PIPELINED, 0), (pstd.XY_CLUSTER, 0, 0), (3, 0, 0),
                    (pstd.XY_SEPARATE, pstd.LINE_TMA, 0), (pstd.XY_SEPARATE, 0, pstd.LINE_PIPELINED),
                    (pstd.XY_SEPARATE, 0, 0, 0b001)):
            with pytest.raises(pstd.PstdError) as e:
                g.set_variants(*bad)
            assert e.value.code == "EINVAL"


def test_bounded_wait_gives_up_and_the_context_survives():
    # the time-bounded mbarrier wait of the TMA-fed passes, on a barrier nothing arrives on
    status, waited = pstd.selftest_bounded_wait(0.05)
    assert status == "ETIMEOUT" and 0.05 <= waited < 1.0
    assert pstd.selftest_bounded_wait(2.0)[0] == "EINVAL"          # limits above a second are refused
    # the context still runs the step kernels afterwards
    spec = ONE_STEP_SPECS["line256-z"]("exact")
    V = random_core_V(spec, 3)
    prev = inputs.random_field(spec.shape, 5)
    cur = inputs.random_field(spec.shape, 6)
    sim = po.Simulation(spec, V, (0.3, -0.5, 0.81), K, 0.05)
    sim.prev, sim.cur, sim.n = prev.copy(), cur.copy(), 17
    sim.step(1)
    with pstd.Grid(spec, precision=pstd.F32) as g:
        g.set_variants(pstd.XY_SEPARATE, pstd.LINE_PLAIN, pstd.LINE_TMA)
        g.set_potential(V)
        g.set_incidence(0, (0.3, -0.5, 0.81), K, 0.05)
        g.set_field(0, prev.astype(np.complex64), cur.astype(np.complex64), 17)
        g.step(1)
        g.synchronize()
        assert rel(g.get_field(0), sim.cur) < 2e-6
