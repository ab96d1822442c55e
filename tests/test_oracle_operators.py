"""Pins of the FP64 oracle's operators against closed forms and the paper's printed values.

CPU only.  Every check compares the oracle with something other than itself: an
exact eigen-relation, a closed-form leapfrog evolution, a property the paper states,
or a number the paper prints (tests/golden/paper_values.json).
"""
import json
import math
import os

import numpy as np
import pytest

from oracle import analytic as an
from oracle import pstd_oracle as po
from paper_2403_04053_gb300 import inputs

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def _periodic_spec(n=(16, 16, 16), d=(0.25, 0.25, 0.25), dt=0.004):
    # no absorber, V = 0: a periodic box on which Fourier modes are exact eigenfunctions
    lo = tuple(m // 4 for m in n)
    hi = tuple(m - m // 4 for m in n)
    return inputs.GridSpec(n=n, d=d, dt=dt, abc_cells=(0, 0, 0), tfsf_lo=lo, tfsf_hi=hi, taper_cells=1,
                           huygens_lo=tuple(v - 1 for v in lo), huygens_hi=tuple(v + 1 for v in hi))


def _mode(spec, m):
    x = [po.coords(spec.n[a], spec.d[a]) for a in range(3)]
    k = [2 * math.pi * m[a] / (spec.n[a] * spec.d[a]) for a in range(3)]
    Z, Y, X = np.meshgrid(x[2], x[1], x[0], indexing="ij")
    return np.exp(1j * (k[0] * X + k[1] * Y + k[2] * Z)), np.array(k)


@pytest.mark.parametrize("n", [12, 16, 48])
def test_kinetic_eigenvalues_on_every_fourier_mode(n):
    """K e^{i k.r} = |k|^2 e^{i k.r} for every grid mode, Nyquist included (Eq. spatialFFTeigen)."""
    spec = _periodic_spec(n=(n, 8, 6), d=(0.3, 0.25, 0.2))
    for m in [(0, 0, 0), (1, 0, 0), (-n // 2, 0, 0), (n // 2 - 1, 3, -2), (-3, -4, 3), (2, 1, -3)]:
        u, k = _mode(spec, m)
        Ku = po.kinetic(u, spec.d)
        assert np.max(np.abs(Ku - (k @ k) * u)) < 1e-10 * max(1.0, k @ k)


def test_kinetic_is_minus_laplacian_on_smooth_periodic_field():
    """-laplacian of exp(sin(2 pi x/L) + cos(2 pi y/L)) in closed form, to spectral accuracy."""
    spec = _periodic_spec(n=(48, 32, 8), d=(0.25, 0.375, 1.0))
    x = [po.coords(spec.n[a], spec.d[a]) for a in range(3)]
    Lx, Ly = spec.n[0] * spec.d[0], spec.n[1] * spec.d[1]
    Z, Y, X = np.meshgrid(x[2], x[1], x[0], indexing="ij")
    ax, ay = 2 * math.pi / Lx, 2 * math.pi / Ly
    f = np.exp(np.sin(ax * X) + np.cos(ay * Y))
    lap = f * ((ax * np.cos(ax * X)) ** 2 - ax * ax * np.sin(ax * X) + (ay * np.sin(ay * Y)) ** 2 - ay * ay * np.cos(ay * Y))
    assert np.max(np.abs(po.kinetic(f.astype(complex), spec.d) + lap)) < 1e-9 * np.max(np.abs(lap))
    dfx = f * ax * np.cos(ax * X)
    assert np.max(np.abs(po.derivative(f.astype(complex), 0, spec.d[0]) - dfx)) < 1e-10 * np.max(np.abs(dfx))


def test_derivative_of_nyquist_mode_uses_literal_index():
    """i k with k = -pi/d at the Nyquist index (literal -N/2..N/2-1 range)."""
    spec = _periodic_spec(n=(8, 8, 8))
    u, k = _mode(spec, (-4, 0, 0))
    assert np.max(np.abs(po.derivative(u, 0, spec.d[0]) - 1j * k[0] * u)) < 1e-12


def test_eta_corrected_leapfrog_is_exact_at_the_carrier_energy():
    """A grid mode with |k| = k0 keeps the physical phase e^{-i E0 t/hbar} for 2000 steps (Eq. numdis2)."""
    spec = _periodic_spec()
    u, kv = _mode(spec, (4, 0, 0))            # k = 2 pi at L = 4
    k0 = float(np.linalg.norm(kv))
    sim = po.Simulation(spec, np.zeros(spec.shape), (1, 0, 0), k0, 0.0)
    w0 = k0 * k0 / 2
    sim.prev = u * np.exp(1j * w0 * spec.dt)
    sim.cur = u.copy()
    nsteps = 2000
    sim.step(nsteps)
    exact = u * np.exp(-1j * w0 * nsteps * spec.dt)
    assert np.max(np.abs(sim.cur - exact)) < 1e-10
    # without eta the same mode drifts in phase: the correction is doing the work
    assert abs(po.eta(w0, spec.dt) - 1.0) > 1e-4


def test_leapfrog_follows_closed_form_for_an_off_carrier_mode():
    """Oblique mode with |k| != k0: psi^n = e^{-i w n dt}, sin(w dt) = dt eta |k|^2 / 2 (Eq. q_equation)."""
    spec = _periodic_spec()
    u, kv = _mode(spec, (1, 2, -3))
    k0 = 2 * math.pi
    sim = po.Simulation(spec, np.zeros(spec.shape), (0, 0, 1), k0, 0.0)
    w = an.leapfrog_mode_frequency(kv @ kv, spec.dt, sim.eta)
    sim.prev = u * np.exp(1j * w * spec.dt)
    sim.cur = u.copy()
    sim.step(1500)
    assert np.max(np.abs(sim.cur - u * np.exp(-1j * w * 1500 * spec.dt))) < 1e-10


def test_unstable_dt_grows_at_the_joukowsky_rate():
    """Above the bound of Eq. PSTDstability the corner mode grows by |Q| = w + sqrt(w^2 - 1) per step."""
    spec = _periodic_spec(n=(8, 8, 8))
    spec.dt = 1.2 * po.stability_dt_max(spec.n, spec.d, 0.0)
    u, kv = _mode(spec, (-4, -4, -4))
    sim = po.Simulation(spec, np.zeros(spec.shape), (0, 0, 1), 2 * math.pi, 0.0)
    sim.cur = u.copy()
    norms = []
    for _ in range(60):
        sim.step()
        norms.append(np.max(np.abs(sim.cur)))
    ratio = norms[-1] / norms[-2]
    assert ratio == pytest.approx(an.leapfrog_growth(kv @ kv, spec.dt, sim.eta), rel=1e-8)
    assert ratio > 1.5


def test_stability_bound_admits_the_papers_time_step():
    """The paper's dtau = pi/1000 at dx_bar = pi/10 satisfies Eq. dtau_stability for |V| <= E0, tightly."""
    g = GOLDEN["stability_example"]
    dx = g["dx_bar_over_pi"] * math.pi         # k0 = 1, so x_bar = x
    E0 = 0.5                                    # hbar = m = k0 = 1
    dtau = g["dtau_over_pi"] * math.pi
    for s in g["s_values"]:
        dtau_max = E0 * po.stability_dt_max((1, 1, 1), (dx, dx, dx), abs(s) * E0)
        assert dtau <= dtau_max
        assert dtau / dtau_max > 0.9           # the paper sits just inside its bound


def test_first_step_of_config_one_is_rejected_as_unstable():
    """dt = 0.005 at dx = 0.25 with V0 = 0.3 E0 is above the bound 0.004119 (so the 48^3 case runs at 0.004)."""
    E0 = 2 * math.pi ** 2
    bound = po.stability_dt_max((48,) * 3, (0.25,) * 3, 0.3 * E0)
    assert bound == pytest.approx(0.004119, abs=2e-6)
    assert 0.005 > bound > 0.004


def test_taper_xi_properties_stated_in_the_paper():
    """xi(0)=0, xi(1)=1 and derivatives 1..4 vanish at both ends (Eq. xi); dxi, d2xi match finite differences."""
    g = GOLDEN["taper_properties"]
    assert po.xi(0.0) == pytest.approx(0.0, abs=1e-15)
    assert po.xi(1.0) == pytest.approx(1.0, abs=1e-15)
    h = 1e-3
    for x0 in (0.0, 1.0):
        f = lambda t: po.xi(x0 + t)
        d1 = (f(-2 * h) - 8 * f(-h) + 8 * f(h) - f(2 * h)) / (12 * h)
        d2 = (-f(-2 * h) + 16 * f(-h) - 30 * f(0) + 16 * f(h) - f(2 * h)) / (12 * h * h)
        d3 = (-f(-2 * h) + 2 * f(-h) - 2 * f(h) + f(2 * h)) / (2 * h ** 3)
        d4 = (f(-2 * h) - 4 * f(-h) + 6 * f(0) - 4 * f(h) + f(2 * h)) / h ** 4
        scale = (2 * math.pi) ** np.array([1, 2, 3, 4])
        vals = dict(zip([1, 2, 3, 4], np.abs([d1, d2, d3, d4]) / scale))
        for order in g["vanishing_derivative_orders"]:
            assert vals[order] < 1e-3, (x0, order, vals[order])
    rho = np.linspace(0.05, 0.95, 19)
    fd1 = (po.xi(rho + 1e-5) - po.xi(rho - 1e-5)) / 2e-5
    fd2 = (po.xi(rho + 1e-4) - 2 * po.xi(rho) + po.xi(rho - 1e-4)) / 1e-8
    assert np.max(np.abs(po.dxi(rho) - fd1)) < 1e-8
    assert np.max(np.abs(po.d2xi(rho) - fd2)) < 1e-4


def test_paper_source_equals_product_rule_of_the_taper():
    """hbar^2/2m (lap(zeta) psi_inc + 2 grad zeta . grad psi_inc) = hbar^2/2m (lap(zeta psi_inc) - zeta lap psi_inc)
    (the step leading to Eq. tildeSchrodinger), with the right side by finite differences."""
    n = 48
    spec = inputs.GridSpec(n=(n, n, n), d=(0.25,) * 3, dt=0.004, tfsf_lo=(12,) * 3, tfsf_hi=(36,) * 3,
                           taper_cells=8, huygens_lo=(10,) * 3, huygens_hi=(38,) * 3, tfsf_mode="paper")
    khat = np.array([0.36, 0.48, 0.8])
    sim = po.Simulation(spec, np.zeros(spec.shape), khat, 2 * math.pi, 0.0)
    src = sim.src_factor * sim.inc_phase
    # fine 1-D sampling along a line through the transition layer, 4th-order differences
    h = 1e-3
    for a, (j, k) in [(0, (20, 24)), (1, (17, 30)), (2, (24, 15))]:
        for i in range(13, 20):
            idx = [j, k]
            idx.insert(a, i)
            r0 = np.array([po.coords(n, 0.25)[t] for t in idx])

            def F(r):
                z = 1.0
                for b in range(3):
                    zz, _, _ = _zeta_at(spec, b, r[b])
                    z *= zz
                return z * np.exp(1j * 2 * math.pi * khat @ (r - sim.rO))

            def Zeta(r):
                z = 1.0
                for b in range(3):
                    z *= _zeta_at(spec, b, r[b])[0]
                return z

            lapF = 0.0
            for b in range(3):
                e = np.zeros(3)
                e[b] = h
                lapF += (-F(r0 + 2 * e) + 16 * F(r0 + e) - 30 * F(r0) + 16 * F(r0 - e) - F(r0 - 2 * e)) / (12 * h * h)
            lap_inc = -(2 * math.pi) ** 2 * np.exp(1j * 2 * math.pi * khat @ (r0 - sim.rO))
            ref = 0.5 * (lapF - Zeta(r0) * lap_inc)
            got = src[idx[2], idx[1], idx[0]]
            assert abs(got - ref) < 2e-5 * max(1.0, abs(ref)), (a, i, got, ref)


def _zeta_at(spec, axis, x):
    """zeta along one axis at a continuous coordinate (Eq. zeta_y), for finite differences."""
    d = spec.d[axis]
    lo, hi, t = spec.tfsf_lo[axis], spec.tfsf_hi[axis], spec.taper_cells
    y0, y1 = (lo - spec.n[axis] // 2) * d, (lo + t - spec.n[axis] // 2) * d
    y2, y3 = (hi - t - spec.n[axis] // 2) * d, (hi - spec.n[axis] // 2) * d
    if x <= y0 or x >= y3:
        return 0.0, 0.0, 0.0
    if x < y1:
        return float(po.xi((x - y0) / (y1 - y0))), 0.0, 0.0
    if x <= y2:
        return 1.0, 0.0, 0.0
    return float(1.0 - po.xi((x - y2) / (y3 - y2))), 0.0, 0.0


def test_first_contact_corner_is_the_box_corner_met_first():
    """O minimises khat . r over the TF/SF box; it agrees with Eq. Oinc wherever that equation is consistent."""
    spec = inputs.square_barrier_workload(with_outputs=False).spec
    lo = po.coords(48, 0.25)[14]
    hi = po.coords(48, 0.25)[34]
    rng = np.random.default_rng(7)
    for _ in range(200):
        kh = rng.standard_normal(3)
        kh /= np.linalg.norm(kh)
        O = po.first_contact_corner(kh, spec)
        corners = np.array([[x, y, z] for x in (lo, hi) for y in (lo, hi) for z in (lo, hi)])
        assert np.all(corners @ kh >= O @ kh - 1e-12)
        th, ph = math.acos(kh[2]), math.atan2(kh[1], kh[0]) % (2 * math.pi)
        zO = lo if th <= math.pi / 2 else hi
        if ph <= math.pi / 2:                       # Eq. Oinc case (i0, j0)
            assert tuple(O) == (lo, lo, zO)
        elif math.pi < ph <= 1.5 * math.pi:         # case (i1, j1)
            assert tuple(O) == (hi, hi, zO)
        elif math.pi / 2 < ph <= math.pi:           # printed (i0, j1); k_x < 0, k_y > 0 meet (i1, j0) first
            assert tuple(O) == (hi, lo, zO)
        else:                                       # printed (i1, j0); k_x > 0, k_y < 0 meet (i0, j1) first
            assert tuple(O) == (lo, hi, zO)


def test_running_dft_is_the_closed_form_geometric_sum():
    """acc = sum_n A e^{-i W t_n} e^{i w t_n} (Eq. psiphasor); the normal derivative sum is i k_x times it."""
    spec = _periodic_spec()
    u, kv = _mode(spec, (2, 0, 0))
    W = 17.3
    w = 2 * math.pi ** 2
    n0, M = 37, 91
    sim = po.Simulation(spec, np.zeros(spec.shape), (1, 0, 0), 2 * math.pi, 0.0, window=(n0, M))
    for n in range(n0, n0 + M):
        sim.n = n
        sim.cur = u * np.exp(-1j * W * n * spec.dt)
        sim.accumulate()
    x = (w - W) * spec.dt
    geo = np.exp(1j * x * n0) * (1 - np.exp(1j * x * M)) / (1 - np.exp(1j * x))
    for face, (a, s) in enumerate(po.FACES):
        h = spec.huygens_lo[a] if s == 0 else spec.huygens_hi[a]
        expect = po.plane_slice(u, a, h) * geo
        assert np.max(np.abs(sim.acc_psi[0][face] - expect)) < 1e-11 * M
        dexp = 1j * kv[a] * expect
        assert np.max(np.abs(sim.acc_dpsi[0][face] - dexp)) < 1e-10 * M
    # incident phasor at O: sum a(t_n) e^{-i w0 t_n} e^{i w t_n} = M at w = w0 once the ramp is over
    assert sim.acc_inc[0] == pytest.approx(M, rel=1e-12)


def test_exact_form_injects_nothing_when_V_is_zero():
    """Zero scattered-field leakage at V = 0 in the exact TF/SF form: the state stays identically 0."""
    wl = inputs.square_barrier_workload(with_outputs=False)
    sim = po.Simulation(wl.spec, np.zeros(wl.spec.shape), (0.36, 0.48, 0.8), 2 * math.pi, 0.5)
    sim.step(200)
    assert np.count_nonzero(sim.cur) == 0 and np.count_nonzero(sim.prev) == 0


def test_absorber_removes_an_outgoing_packet():
    """A packet run into the masking layer (Eqs. expmask, Gamma) leaves < 1e-4 of its norm in the free region."""
    spec = inputs.GridSpec(n=(8, 8, 256), d=(0.25,) * 3, dt=0.004, abc_cells=(0, 0, 24),
                           tfsf_lo=(2, 2, 100), tfsf_hi=(6, 6, 156), taper_cells=1,
                           huygens_lo=(1, 1, 90), huygens_hi=(7, 7, 166))
    z = po.coords(256, 0.25)
    k0 = 2 * math.pi
    sim = po.Simulation(spec, np.zeros(spec.shape), (0, 0, 1), k0, 0.0)
    w0 = k0 * k0 / 2

    def packet(t):
        # free Gaussian packet e^{i(k0 z - w0 t)} with centre z0 + k0 t (spreading is slow at sigma = 2)
        env = np.exp(-((z + 10.0 - k0 * t) ** 2) / (2 * 2.0 ** 2))
        return (env * np.exp(1j * (k0 * z - w0 * t)))[:, None, None] * np.ones((1, 8, 8))

    sim.prev = packet(-spec.dt)
    sim.cur = packet(0.0)
    free = slice(24, 232)
    norm0 = np.sum(np.abs(sim.cur[free]) ** 2)
    sim.step(2400)        # t = 9.6: the packet centre has gone 60 units, through the layer
    assert np.sum(np.abs(sim.cur[free]) ** 2) < 1e-4 * norm0
