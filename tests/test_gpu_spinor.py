"""GPU parity of spinor grids (pstd_set_magnetic_field) against the FP64 spinor oracle.

A spinor grid pairs its batch members (2p, 2p + 1) as the up and down components coupled by
W = V I + gamma sigma . B.  Tolerances are those of the scalar path (the coupling adds one
complex product per node): FP64 1e-12 after one step, FP32 2e-6; short runs 1e-12 / 2e-5 on the
state, ten times that on phasors, 1e-10 / 2e-4 on transforms and cross-sections.
"""
import math

import numpy as np
import pytest

from oracle import ntdf_oracle as no
from oracle import spinor_oracle as so
from paper_2403_04053_gb300 import inputs, pstd

pytestmark = pytest.mark.gpu

K = 2 * math.pi
KHAT = (0.3, -0.5, 0.81)
CHI = (0.6, 0.8j)


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def ragged_spec(mode="exact"):
    return inputs.GridSpec(n=(24, 32, 48), d=(0.25, 0.3, 0.2), dt=0.002, abc_cells=(4, 5, 6), tfsf_lo=(9, 12, 17),
                           tfsf_hi=(15, 20, 31), taper_cells=2, huygens_lo=(7, 9, 14), huygens_hi=(17, 23, 34),
                           tfsf_mode=mode)


def square_spec():
    # square planes: the fused x+y pass
    return inputs.GridSpec(n=(64, 64, 48), d=(0.25, 0.25, 0.3), dt=0.002, abc_cells=(6, 6, 5), tfsf_lo=(20, 20, 16),
                           tfsf_hi=(44, 44, 32), taper_cells=3, huygens_lo=(14, 14, 10), huygens_hi=(50, 50, 38))


def core_fields(spec, seed, vamp=2.0, bamp=3.0, b_shrink=0):
    """Random V and a random-direction B on the zeta == 1 core (B on a box shrunk by b_shrink)."""
    rng = np.random.default_rng(seed)
    c = spec.core_box()
    sl = tuple(slice(c[a][0], c[a][1] + 1) for a in (2, 1, 0))
    V = np.zeros(spec.shape)
    V[sl] = rng.uniform(-vamp, vamp, V[sl].shape)
    B = [np.zeros(spec.shape) for _ in range(3)]
    bl = tuple(slice(c[a][0] + b_shrink, c[a][1] + 1 - b_shrink) for a in (2, 1, 0))
    for comp in B:
        comp[bl] = rng.uniform(-bamp, bamp, comp[bl].shape)
    return V, B


def spinor_grid(spec, prec, V, B, gamma, batch=2):
    g = pstd.Grid(spec, precision=prec, batch=batch)
    g.set_potential(V)
    g.set_magnetic_field(B, gamma)
    return g


@pytest.mark.parametrize("prec,tol", [(pstd.F64, 1e-12), (pstd.F32, 2e-6)])
@pytest.mark.parametrize("which", ["ragged", "square", "b-box-only"])
def test_one_step_matches_spinor_oracle(which, prec, tol):
    spec = square_spec() if which == "square" else ragged_spec()
    V, B = core_fields(spec, 3, b_shrink=1)
    if which == "b-box-only":
        V = np.zeros(spec.shape)        # the source region is B's box alone
    gamma = 1.3
    prev = [inputs.random_field(spec.shape, 5 + s) for s in range(2)]
    cur = [inputs.random_field(spec.shape, 7 + s) for s in range(2)]
    sim = so.SpinorSimulation(spec, V, B, gamma, KHAT, K, 0.05, CHI)
    for s in range(2):
        sim.comp[s].prev, sim.comp[s].cur, sim.comp[s].n = prev[s].copy(), cur[s].copy(), 17
    sim.n = 17
    sim.step(1)
    cd = np.complex128 if prec == pstd.F64 else np.complex64
    with spinor_grid(spec, prec, V, B, gamma) as g:
        g.set_incidence_spinor(0, KHAT, K, 0.05, CHI)
        for s in range(2):
            g.set_field(s, prev[s].astype(cd), cur[s].astype(cd), 17)
        g.step(1)
        for s in range(2):
            assert rel(g.get_field(s), sim.cur[s]) < tol


@pytest.fixture(scope="module")
def spinor_run():
    spec = ragged_spec()
    V, B = core_fields(spec, 11)
    gamma = 1.1
    w0 = K * K / 2
    om = [w0, 0.93 * w0]
    win = (20, 40)
    sim = so.SpinorSimulation(spec, V, B, gamma, KHAT, K, 0.05, CHI, window=win, omegas=om)
    sim.step(60)
    pts = np.array([[3.0, -2.0, 5.5], [-4.0, 6.0, 1.0], [30.0, 10.0, 40.0], [-200.0, 50.0, 120.0]])
    th = np.deg2rad(np.array([0.0, 33.0, 90.0, 140.0, 180.0]))
    ph = np.deg2rad(np.array([0.0, 20.0, 200.0, 300.0, 10.0]))
    ref = {}
    for s in range(2):
        for f in range(2):
            k = math.sqrt(2 * om[f])
            phs = sim.scaled_phasors(s, f)
            ref[s, f] = (phs, no.transform_to_points(spec, k, phs, pts), no.cross_section(spec, k, phs, th, ph))
    return dict(spec=spec, V=V, B=B, gamma=gamma, om=om, win=win, sim=sim, pts=pts, th=th, ph=ph, ref=ref)


@pytest.mark.parametrize("prec,tol_state,tol_out", [(pstd.F64, 1e-12, 1e-10), (pstd.F32, 2e-5, 2e-4)])
def test_short_run_spin_resolved_outputs(spinor_run, prec, tol_state, tol_out):
    r = spinor_run
    with spinor_grid(r["spec"], prec, r["V"], r["B"], r["gamma"]) as g:
        g.set_incidence_spinor(0, KHAT, K, 0.05, CHI)
        g.huygens_dft(-1, r["om"], *r["win"])
        g.step(60)
        for s in range(2):
            assert rel(g.get_field(s), r["sim"].cur[s]) < tol_state
            for f in range(2):
                phs, psi_ref, (ds_ref, f_ref) = r["ref"][s, f]
                for (gp, gd), (rp, rd) in zip(g.get_phasors(s, f), phs):
                    assert rel(gp, rp) < 10 * tol_state and rel(gd, rd) < 10 * tol_state
                psi = g.transform_to_points(s, f, r["pts"])
                assert np.max(np.abs(psi - psi_ref) / np.abs(psi_ref)) < tol_out
                ds, fa = g.cross_section(s, f, r["th"], r["ph"])
                assert np.max(np.abs(fa - f_ref) / np.abs(f_ref)) < tol_out
                assert np.max(np.abs(ds - ds_ref) / ds_ref) < 2 * tol_out


def test_spin_flip_needs_the_transverse_field():
    # an up-polarised wave on B = Bz zhat stays up (the down component is exactly zero);
    # a transverse Bx flips part of it
    spec = ragged_spec()
    V, B = core_fields(spec, 4)
    Bz_only = [np.zeros(spec.shape), np.zeros(spec.shape), B[2]]
    for field, flips in ((Bz_only, False), (B, True)):
        with spinor_grid(spec, pstd.F32, V, field, 1.2) as g:
            g.set_incidence_spinor(0, KHAT, K, 0.05, (1.0, 0.0))
            g.step(40)
            up, dn = g.get_field(0), g.get_field(1)
            assert np.linalg.norm(up) > 0
            if flips:
                assert np.linalg.norm(dn) > 1e-3 * np.linalg.norm(up)
            else:
                assert not np.any(dn)


def test_spinor_pairs_in_one_batch_equal_separate_grids():
    spec = ragged_spec()
    V, B = core_fields(spec, 5)
    cases = [(KHAT, CHI), ((-0.6, 0.0, 0.8), (1.0, 0.0))]
    w0 = K * K / 2
    outs = []
    for kh, chi in cases:
        with spinor_grid(spec, pstd.F32, V, B, 0.9) as g:
            g.set_incidence_spinor(0, kh, K, 0.05, chi)
            g.huygens_dft(-1, [w0], 10, 20)
            g.step(30)
            outs.append([(g.get_field(s), g.transform_to_points(s, 0, [[5.0, 5.0, 9.0]])) for s in range(2)])
    with spinor_grid(spec, pstd.F32, V, B, 0.9, batch=4) as g:
        for p, (kh, chi) in enumerate(cases):
            g.set_incidence_spinor(p, kh, K, 0.05, chi)
        g.huygens_dft(-1, [w0], 10, 20)
        g.step(30)
        for p in range(2):
            for s in range(2):
                assert np.array_equal(g.get_field(2 * p + s), outs[p][s][0])
                assert np.array_equal(g.transform_to_points(2 * p + s, 0, [[5.0, 5.0, 9.0]]), outs[p][s][1])


def test_graph_replay_on_a_spinor_grid():
    spec = square_spec()
    V, B = core_fields(spec, 6)
    res = []
    for graphs in (False, True):
        with spinor_grid(spec, pstd.F32, V, B, 1.0) as g:
            g.set_graphs(graphs)
            g.set_incidence_spinor(0, KHAT, K, 0.05, CHI)
            g.huygens_dft(-1, [K * K / 2], 5, 10)
            for _ in range(3):
                g.reset()
                g.step(20)
            res.append([g.get_field(s) for s in range(2)] + [g.graph_replays()])
    assert res[0][2] == 0 and res[1][2] == 2
    for s in range(2):
        assert np.array_equal(res[0][s], res[1][s])


def test_spinor_call_errors():
    spec = ragged_spec()
    V, B = core_fields(spec, 7)
    with pstd.Grid(spec, precision=pstd.F32, batch=3) as g:           # odd batch
        with pytest.raises(pstd.PstdError) as e:
            g.set_magnetic_field(B, 1.0)
        assert e.value.code == "EINVAL"
    with pstd.Grid(ragged_spec("paper"), precision=pstd.F32, batch=2) as g:   # PAPER form
        with pytest.raises(pstd.PstdError) as e:
            g.set_magnetic_field(B, 1.0)
        assert e.value.code == "EINVAL"
    with pstd.Grid(spec, precision=pstd.F32, batch=2) as g:
        outside = [b.copy() for b in B]
        outside[1][0, 0, 0] = 1.0                                        # B in the absorbing layer
        with pytest.raises(pstd.PstdError) as e:
            g.set_magnetic_field(outside, 1.0)
        assert e.value.code == "EINVAL"
        with pytest.raises(pstd.PstdError) as e:
            g.set_magnetic_field(B, 1e6)                                # |gamma B| breaks the dt bound
        assert e.value.code == "EUNSTABLE"
        g.set_magnetic_field(B, 1.0)
        with pytest.raises(pstd.PstdError) as e:
            g.set_incidence(0, KHAT, K, 0.05)                           # scalar incidence on a spinor grid
        assert e.value.code == "EINVAL"
        with pytest.raises(pstd.PstdError) as e:
            g.set_incidence_packet(0, KHAT, K, 1.0, -3.0)
        assert e.value.code == "EINVAL"
        with pytest.raises(pstd.PstdError) as e:
            g.set_incidence_spinor(1, KHAT, K, 0.05, CHI)               # spinor 1 needs members 2, 3
        assert e.value.code == "EINVAL"
        # |V|max = 240 alone is within the bound 1/dt - kinetic = 242.8 of this grid, not with |gamma B|max
        Vbig = V * (240.0 / np.abs(V).max())
        assert np.sqrt(sum(b ** 2 for b in B)).max() > 3.0
        with pytest.raises(pstd.PstdError) as e:
            g.set_potential(Vbig)
        assert e.value.code == "EUNSTABLE"
    with pstd.Grid(spec, precision=pstd.F32, batch=2) as g:
        g.set_potential(Vbig)                                           # stable without B


# ----------------------------------------------------------------------------------
# the 384^3 point-dipole configuration at full size, in the bench's launch configuration
# (two spinors = four members, FP32): sampled nodes against the node-by-node oracle
# ----------------------------------------------------------------------------------
@pytest.fixture(scope="module")
def dipole():
    return inputs.spinor_workload(with_outputs=True)


def _dipole_grid(wl):
    g = pstd.Grid(wl.spec, precision=pstd.F32, batch=2 * len(wl.chis))
    g.set_potential(wl.V)
    g.set_magnetic_field(wl.B, wl.gamma)
    inc = wl.incidences[0]
    for p, chi in enumerate(wl.chis):
        g.set_incidence_spinor(p, inc.khat, inc.k, inc.ramp_time, chi)
    return g


def test_384_cubed_spinor_one_step_sampled(dipole):
    wl = dipole
    sp, inc = wl.spec, wl.incidences[0]
    n = 300                                     # past the ramp: the full incident amplitude
    prev = [inputs.random_field_c64(sp.shape, 40 + b) for b in range(4)]
    cur = [inputs.random_field_c64(sp.shape, 50 + b) for b in range(4)]
    rng = np.random.default_rng(12)
    nodes = [(0, 0, 0), (383, 383, 383), (5, 200, 379), (192, 192, 192), (150, 240, 145), (239, 145, 200),
             (130, 130, 130), (253, 128, 190)]
    nodes += [tuple(int(v) for v in rng.integers(0, 384, 3)) for _ in range(24)]          # anywhere
    nodes += [tuple(int(v) for v in rng.integers(145, 240, 3)) for _ in range(24)]        # inside B's support
    with _dipole_grid(wl) as g:
        for b in range(4):
            g.set_field(b, prev[b], cur[b], n)
        g.step(1)
        got = [g.get_field(b) for b in range(4)]
    for p, chi in enumerate(wl.chis):
        ref = so.step_at_nodes(sp, wl.V, wl.B, wl.gamma, inc.khat, inc.k, inc.ramp_time, chi,
                               prev[2 * p:2 * p + 2], cur[2 * p:2 * p + 2], n, nodes)
        scale = np.max(np.abs(ref))
        for q, (i, j, k) in enumerate(nodes):
            for s in range(2):
                assert abs(got[2 * p + s][k, j, i] - ref[q, s]) < 4e-5 * scale


def test_384_cubed_spinor_sampled_transform(dipole):
    """Phasors of a short full-size run; the transform at a sampled Fresnel-plane point (spin-flip
    members) and the far field at sampled directions (every member) against the oracle's mode
    sums on the GPU's own phasors."""
    wl = dipole
    w0 = K * K / 2
    with _dipole_grid(wl) as g:
        g.huygens_dft(-1, [w0], 30, 30)
        g.step(60)
        phs = [g.get_phasors(b, 0) for b in range(4)]
        pt = wl.fresnel_points[[131000]]
        psi = {b: g.transform_to_points(b, 0, pt) for b in (1, 2)}
        th = np.deg2rad([5.0, 91.0, 170.0])
        ph = np.deg2rad([10.0, 250.0, 0.0])
        far = [g.cross_section(b, 0, th, ph)[1] for b in range(4)]
    for b in (1, 2):
        ref = no.transform_to_points(wl.spec, K, phs[b], pt)
        assert np.max(np.abs(psi[b] - ref) / np.abs(ref)) < 1e-4
    for b in range(4):
        _, fref = no.cross_section(wl.spec, K, phs[b], th, ph)
        assert np.max(np.abs(far[b] - fref) / np.abs(fref)) < 1e-4

