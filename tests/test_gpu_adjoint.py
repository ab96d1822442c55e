"""GPU discrete adjoint against the FP64 oracle's adjoint and against finite differences.

Tolerances (relative, from the arithmetic): FP64 path 1e-9 (the G = 8 cell quadrature
reproduces the oracle's sinc sum to ~1e-13; the backward sweep adds round-off of the
same order as the forward run); FP32 path 2e-4 on the transform adjoint and 2e-3 on
dL/dV (single-precision round-off accumulated over the forward and the backward sweep,
ten times the FP32 state tolerance); finite differences 1e-6 (central differences with
h = 1e-4 in FP64).
"""
import math

import numpy as np
import pytest

from oracle import adjoint_oracle as ao
from paper_2403_04053_gb300 import inputs, pstd

pytestmark = pytest.mark.gpu

K = 2 * math.pi
E0 = 0.5 * K * K
KHAT = (0.3, -0.5, 0.81)
PTS = np.array([[3.0, -2.0, 5.5], [-4.0, 6.0, 1.0], [0.5, 0.2, -9.0], [1.0, 2.0, 3.0]])
TARGET = np.full(len(PTS), 0.01)
NSTEPS, WIN = 80, (50, 30)


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


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


def gpu_forward(spec, V, prec, nsteps=NSTEPS, win=WIN):
    g = pstd.Grid(spec, precision=prec)
    g.set_potential(V)
    g.set_incidence(0, KHAT, K, 0.05)
    g.huygens_dft(0, [E0], *win)
    g.step(nsteps)
    psi = g.transform_to_points(0, 0, PTS)
    L, gpts = ao.magnitude_misfit(psi, TARGET)
    return g, psi, L, gpts


def box_of(spec, mode):
    if mode == "exact":
        return (2, 2, 2), (22, 22, 22)          # beyond the core too, where V itself must vanish
    c = spec.core_box()
    return tuple(c[a][0] for a in range(3)), tuple(c[a][1] + 1 for a in range(3))


def sub(arr, lo, hi):
    return arr[lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]]


@pytest.mark.parametrize("prec,tol", [(pstd.F64, 1e-9), (pstd.F32, 2e-4)])
def test_transform_adjoint_matches_oracle(prec, tol):
    spec = small_spec("exact")
    rng = np.random.default_rng(2)
    y = rng.standard_normal(len(PTS)) + 1j * rng.standard_normal(len(PTS))
    with pstd.Grid(spec, precision=prec) as g:
        g.set_incidence(0, KHAT, K, 0.05)
        got = g.transform_adjoint(0, 0, PTS, y)
    ref = ao.transform_adjoint(spec, K, PTS, y)
    assert rel(g.join_phasors(got), g.join_phasors(ref)) < tol


@pytest.mark.parametrize("prec,tol", [(pstd.F64, 1e-9), (pstd.F32, 2e-3)])
@pytest.mark.parametrize("mode", ["exact", "paper"])
def test_adjoint_gradient_matches_oracle(mode, prec, tol):
    spec = small_spec(mode)
    V = core_V(spec, 7)
    L_ref, grad_ref, psi_ref = ao.fresnel_loss_and_gradient(spec, V, KHAT, K, 0.05, WIN, NSTEPS, PTS, TARGET)
    lo, hi = box_of(spec, mode)
    g, psi, L, gpts = gpu_forward(spec, V, prec)
    with g:
        assert rel(psi, psi_ref) < (1e-10 if prec == pstd.F64 else 2e-4)
        g_ph = g.transform_adjoint(0, 0, PTS, gpts)
        grad = g.adjoint_gradient(NSTEPS, [g_ph], lo, hi)
        assert g.get_step() == 0                   # left at rest
    assert rel(grad, sub(grad_ref, lo, hi)) < tol


def test_adjoint_gradient_matches_gpu_finite_differences():
    spec = small_spec("exact")
    V = core_V(spec, 9)
    lo, hi = (2, 2, 2), (22, 22, 22)
    g, psi, L, gpts = gpu_forward(spec, V, pstd.F64)
    with g:
        grad = g.adjoint_gradient(NSTEPS, [g.transform_adjoint(0, 0, PTS, gpts)], lo, hi)
    h = 1e-4
    errs = []
    for (z, y, x) in [(12, 11, 10), (9, 14, 12), (10, 10, 14), (15, 8, 13)]:   # inside the core
        Lpm = []
        for sgn in (1, -1):
            Vp = V.copy()
            Vp[z, y, x] += sgn * h
            gp, _, Lp, _ = gpu_forward(spec, Vp, pstd.F64)
            gp.close()
            Lpm.append(Lp)
        fd = (Lpm[0] - Lpm[1]) / (2 * h)
        errs.append(abs(fd - grad[z - lo[2], y - lo[1], x - lo[0]]))
    assert max(errs) / np.abs(grad).max() < 1e-6


def test_checkpoint_interval_does_not_change_the_gradient():
    spec = small_spec("exact")
    V = core_V(spec, 7)
    g, psi, L, gpts = gpu_forward(spec, V, pstd.F64)
    with g:
        g_ph = g.transform_adjoint(0, 0, PTS, gpts)
        lo, hi = box_of(spec, "exact")
        grads = [g.adjoint_gradient(NSTEPS, [g_ph], lo, hi, k) for k in (0, 1, 7, NSTEPS)]
    for other in grads[1:]:
        assert rel(other, grads[0]) < 1e-13


def test_recorded_checkpoints_give_the_same_gradient():
    # checkpoints recorded by pstd_step replace the adjoint's own forward run; a new
    # potential discards them
    spec = small_spec("exact")
    V1, V2 = core_V(spec, 7), core_V(spec, 8)
    lo, hi = box_of(spec, "exact")
    ref = {}
    for name, V in (("V1", V1), ("V2", V2)):
        g, psi, L, gpts = gpu_forward(spec, V, pstd.F64)
        with g:
            gph = g.transform_adjoint(0, 0, PTS, gpts)
            ref[name] = (gph, g.adjoint_gradient(NSTEPS, [gph], lo, hi, 9))
    with pstd.Grid(spec, precision=pstd.F64) as g:
        g.set_potential(V1)
        g.set_incidence(0, KHAT, K, 0.05)
        g.huygens_dft(0, [E0], *WIN)
        g.set_checkpointing(9, NSTEPS)
        g.reset()
        g.step(NSTEPS)
        assert rel(g.adjoint_gradient(NSTEPS, [ref["V1"][0]], lo, hi, 9), ref["V1"][1]) < 1e-12
        # the same record serves a second call; then a new potential must not reuse it
        assert rel(g.adjoint_gradient(NSTEPS, [ref["V1"][0]], lo, hi, 9), ref["V1"][1]) < 1e-12
        g.set_potential(V2)
        assert rel(g.adjoint_gradient(NSTEPS, [ref["V2"][0]], lo, hi, 9), ref["V2"][1]) < 1e-12


def test_autograd_function_matches_the_adjoint():
    torch = pytest.importorskip("torch")
    spec = small_spec("exact")
    V = core_V(spec, 7)
    lo, hi = box_of(spec, "exact")
    with pstd.Grid(spec, precision=pstd.F64) as g:
        g.set_incidence(0, KHAT, K, 0.05)
        g.huygens_dft(0, [E0], *WIN)
        Vt = torch.tensor(V, device="cuda", requires_grad=True)
        pts = torch.tensor(PTS, device="cuda")
        psi = pstd.fresnel_field(Vt, g, pts, NSTEPS, lo, hi)
        loss = ((psi.abs() - torch.tensor(TARGET, device="cuda")) ** 2).sum()
        loss.backward()
        gV = Vt.grad.cpu().numpy()
    L_ref, grad_ref, _ = ao.fresnel_loss_and_gradient(spec, V, KHAT, K, 0.05, WIN, NSTEPS, PTS, TARGET)
    assert abs(float(loss.detach()) - L_ref) < 1e-9 * L_ref
    assert rel(sub(gV, lo, hi), sub(grad_ref, lo, hi)) < 1e-9
    outside = gV.copy()
    outside[lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]] = 0
    assert not outside.any()


def test_adjoint_call_errors():
    spec = small_spec("exact")
    gph = [np.zeros(1)]
    with pstd.Grid(spec, precision=pstd.F32, batch=2) as g:
        g.set_incidence(0, KHAT, K, 0.05)
        g.huygens_dft(0, [E0], 5, 10)
        with pytest.raises(pstd.PstdError) as e:
            g.adjoint_gradient(20, gph, (0, 0, 0), (4, 4, 4))
        assert e.value.code == "ESTATE"       # member 1 has no incidence
    with pstd.Grid(spec, precision=pstd.F32) as g:
        g.set_incidence(0, KHAT, K, 0.05)
        with pytest.raises(pstd.PstdError) as e:
            g.adjoint_gradient(10, gph, (0, 0, 0), (4, 4, 4))
        assert e.value.code == "ESTATE"       # no DFT window
        g.huygens_dft(0, [E0], 5, 10)
        z = np.zeros(g.phasor_count(), dtype=np.complex128)
        for lo, hi in [((0, 0, 0), (25, 4, 4)), ((3, 0, 0), (3, 4, 4)), ((-1, 0, 0), (4, 4, 4))]:
            with pytest.raises(pstd.PstdError) as e:
                g.adjoint_gradient(20, [z], lo, hi)
            assert e.value.code == "EINVAL"
        with pytest.raises(pstd.PstdError) as e:
            g.adjoint_gradient(12, [z], (0, 0, 0), (4, 4, 4))   # window ends after step 12
        assert e.value.code == "EINVAL"
        # a zero loss gradient gives a zero dL/dV
        assert not g.adjoint_gradient(20, [z], (0, 0, 0), (4, 4, 4)).any()


@pytest.fixture(scope="module")
def oracle_48():
    """The adjoint workload's construction on a 48^3 grid (V on the central 18^3 block of
    seeded smoothed noise, 400 steps, an 8 x 8 Fresnel plane): the FP64 oracle's loss and its
    discrete-adjoint gradient."""
    wl, V_target = inputs.adjoint_workload(n=48, nsteps=400, block=18, fresnel_count=8, abc=4, tf=(8, 40), taper=4,
                                           hb=(5, 43))
    inc = wl.incidences[0]
    win = (wl.window_first, wl.window_len)
    from oracle import ntdf_oracle as no
    from oracle import pstd_oracle as po
    sim = po.Simulation(wl.spec, V_target, inc.khat, inc.k, inc.ramp_time, window=win)
    sim.step(wl.nsteps)
    target = np.abs(no.transform_to_points(wl.spec, inc.k, sim.scaled_phasors(0), wl.fresnel_points))
    L, grad, psi = ao.fresnel_loss_and_gradient(wl.spec, wl.V, inc.khat, inc.k, inc.ramp_time, win, wl.nsteps,
                                                wl.fresnel_points, target)
    return wl, target, L, grad, psi


@pytest.mark.parametrize("prec,tol", [(pstd.F64, 1e-9), (pstd.F32, 2e-3)])
def test_adjoint_gradient_matches_oracle_at_48_cubed(oracle_48, prec, tol):
    wl, target, L_ref, grad_ref, psi_ref = oracle_48
    inc = wl.incidences[0]
    lo, hi = (15, 15, 15), (33, 33, 33)          # the 18^3 block of V
    with pstd.Grid(wl.spec, precision=prec) as g:
        g.set_potential(wl.V)
        g.set_incidence(0, inc.khat, inc.k, inc.ramp_time)
        g.huygens_dft(0, [E0], wl.window_first, wl.window_len)
        g.step(wl.nsteps)
        psi = g.transform_to_points(0, 0, wl.fresnel_points)
        L, gpts = ao.magnitude_misfit(psi, target)
        grad = g.adjoint_gradient(wl.nsteps, [g.transform_adjoint(0, 0, wl.fresnel_points, gpts)], lo, hi)
    assert rel(psi, psi_ref) < (1e-10 if prec == pstd.F64 else 2e-4)
    assert abs(L - L_ref) < (1e-9 if prec == pstd.F64 else 1e-3) * L_ref
    assert rel(grad, sub(grad_ref, lo, hi)) < tol


def test_full_size_adjoint_against_finite_differences():
    # the adjoint workload as stated: 128^3, 2000 steps, V on the central 48^3 block, the |Psi|
    # misfit on a 128 x 128 Fresnel plane against the field of a second seeded potential.
    # Central differences (h = 1e-4, FP64 runs) at 32 seeded voxels of the block against the
    # FP64 adjoint, and the FP32 adjoint against the FP64 one on the whole block
    wl, V_target = inputs.adjoint_workload()
    spec = wl.spec
    inc = wl.incidences[0]
    pts = wl.fresnel_points
    lo, hi = (40, 40, 40), (88, 88, 88)
    win = (wl.window_first, wl.window_len)

    def run(V, prec, target=None):
        g = pstd.Grid(spec, precision=prec)
        g.set_potential(V)
        g.set_incidence(0, inc.khat, inc.k, inc.ramp_time)
        g.huygens_dft(0, [E0], *win)
        g.step(wl.nsteps)
        psi = g.transform_to_points(0, 0, pts)
        if target is None:
            g.close()
            return np.abs(psi)
        L, gpts = ao.magnitude_misfit(psi, target)
        return g, L, gpts

    target = run(V_target, pstd.F64)
    g, L, gpts = run(wl.V, pstd.F64, target)
    with g:
        grad64 = g.adjoint_gradient(wl.nsteps, [g.transform_adjoint(0, 0, pts, gpts)], lo, hi)
    g, L32, gpts32 = run(wl.V, pstd.F32, target)
    with g:
        grad32 = g.adjoint_gradient(wl.nsteps, [g.transform_adjoint(0, 0, pts, gpts32)], lo, hi)
    assert rel(grad32, grad64) < 2e-3
    h = 1e-4
    rng = np.random.default_rng(2407)
    voxels = rng.integers(lo[0], hi[0], size=(32, 3))
    fd, ad = [], []
    for (z, y, x) in voxels:
        Lpm = []
        for sgn in (1, -1):
            V = wl.V.copy()
            V[z, y, x] += sgn * h
            gp, Lp, _ = run(V, pstd.F64, target)
            gp.close()
            Lpm.append(Lp)
        fd.append((Lpm[0] - Lpm[1]) / (2 * h))
        ad.append(grad64[z - lo[2], y - lo[1], x - lo[0]])
    fd, ad = np.array(fd), np.array(ad)
    assert np.max(np.abs(fd - ad)) < 1e-6 * np.abs(grad64).max()
    assert rel(ad, fd) < 1e-5


# two incidences against one V, each along its own direction (the same k: the mask's rate
# is set by member 0's energy, so members of other energies would not match one-member runs)
MEMBERS = ((KHAT, K), ((-0.6, 0.0, 0.8), K))


def batched_forward(spec, V, prec):
    g = pstd.Grid(spec, precision=prec, batch=len(MEMBERS))
    g.set_potential(V)
    for b, (khat, k) in enumerate(MEMBERS):
        g.set_incidence(b, khat, k, 0.05)
        g.huygens_dft(b, [0.5 * k * k], *WIN)
    return g


def member_blocks(g):
    """dL/d(scaled phasors) of every member for L = sum_b sum_p (|Psi_bp| - target_p)^2."""
    blocks, L = [], 0.0
    for b in range(len(MEMBERS)):
        psi = g.transform_to_points(b, 0, PTS)
        Lb, gpts = ao.magnitude_misfit(psi, TARGET)
        L += Lb
        blocks.append(g.transform_adjoint(b, 0, PTS, gpts))
    return L, blocks


@pytest.mark.parametrize("prec,tol", [(pstd.F64, 1e-9), (pstd.F32, 2e-3)])
def test_batched_adjoint_gradient_is_the_sum_over_members(prec, tol):
    # The members share V and the loss adds their misfits, so dL/dV is the sum of each
    # member's discrete-adjoint gradient; the oracle computes each member on its own.
    spec = small_spec("exact")
    V = core_V(spec, 7)
    lo, hi = box_of(spec, "exact")
    L_ref, grad_ref = 0.0, 0.0
    for khat, k in MEMBERS:
        Lb, gb, _ = ao.fresnel_loss_and_gradient(spec, V, khat, k, 0.05, WIN, NSTEPS, PTS, TARGET)
        L_ref, grad_ref = L_ref + Lb, grad_ref + gb
    with batched_forward(spec, V, prec) as g:
        g.step(NSTEPS)
        L, blocks = member_blocks(g)
        grad = g.adjoint_gradient(NSTEPS, blocks, lo, hi)
        assert g.get_step() == 0                   # left at rest
    assert abs(L - L_ref) < (1e-9 if prec == pstd.F64 else 1e-3) * L_ref
    assert rel(grad, sub(grad_ref, lo, hi)) < tol


def test_batched_adjoint_with_recorded_checkpoints():
    # checkpoints of both members recorded by pstd_step give the gradient of the adjoint's
    # own forward run
    spec = small_spec("exact")
    V = core_V(spec, 8)
    lo, hi = box_of(spec, "exact")
    with batched_forward(spec, V, pstd.F64) as g:
        g.step(NSTEPS)
        _, blocks = member_blocks(g)
        own = g.adjoint_gradient(NSTEPS, blocks, lo, hi, 9)
    with batched_forward(spec, V, pstd.F64) as g:
        g.set_checkpointing(9, NSTEPS)
        g.reset()
        g.step(NSTEPS)
        _, blocks = member_blocks(g)
        recorded = g.adjoint_gradient(NSTEPS, blocks, lo, hi, 9)
    assert rel(recorded, own) < 1e-12


def test_adjoint_with_tensor_copy_line_passes():
    # FP32 128-point y and z lines can be fed by tensor copies; their maps cover the grid's
    # own level buffers, so the adjoint levels must take the register-fed passes: the
    # gradient is the same whichever feed the forward run used
    spec = inputs.GridSpec(n=(16, 128, 128), d=(0.25, 0.25, 0.25), dt=0.004, abc_cells=(2, 8, 8), tfsf_lo=(5, 52, 52),
                           tfsf_hi=(11, 76, 76), taper_cells=2, huygens_lo=(3, 48, 48), huygens_hi=(13, 80, 80))
    V = core_V(spec, 3)
    lo, hi = box_of(spec, "paper")              # the core box
    grads = []
    for zmode in (pstd.LINE_PLAIN, pstd.LINE_TMA):
        with pstd.Grid(spec, precision=pstd.F32) as g:
            g.set_variants(pstd.XY_SEPARATE, zmode, zmode)
            g.set_potential(V)
            g.set_incidence(0, KHAT, K, 0.05)
            g.huygens_dft(0, [E0], *WIN)
            g.step(NSTEPS)
            psi = g.transform_to_points(0, 0, PTS)
            _, gpts = ao.magnitude_misfit(psi, TARGET)
            grads.append(g.adjoint_gradient(NSTEPS, [g.transform_adjoint(0, 0, PTS, gpts)], lo, hi))
    assert np.abs(grads[0]).max() > 0
    assert rel(grads[1], grads[0]) < 1e-5


def test_autograd_function_on_a_batch():
    # Psi of both members from one run; the loss over both members backpropagates through
    # the batched adjoint to the sum of the oracle's one-member gradients
    torch = pytest.importorskip("torch")
    spec = small_spec("exact")
    V = core_V(spec, 7)
    lo, hi = box_of(spec, "exact")
    with pstd.Grid(spec, precision=pstd.F64, batch=len(MEMBERS)) as g:
        for b, (khat, k) in enumerate(MEMBERS):
            g.set_incidence(b, khat, k, 0.05)
            g.huygens_dft(b, [0.5 * k * k], *WIN)
        Vt = torch.tensor(V, device="cuda", requires_grad=True)
        pts = torch.tensor(PTS, device="cuda")
        psi = pstd.fresnel_field(Vt, g, pts, NSTEPS, lo, hi)
        assert tuple(psi.shape) == (len(MEMBERS), len(PTS))
        loss = ((psi.abs() - torch.tensor(TARGET, device="cuda")) ** 2).sum()
        loss.backward()
        gV = Vt.grad.cpu().numpy()
    L_ref, grad_ref = 0.0, 0.0
    for khat, k in MEMBERS:
        Lb, gb, _ = ao.fresnel_loss_and_gradient(spec, V, khat, k, 0.05, WIN, NSTEPS, PTS, TARGET)
        L_ref, grad_ref = L_ref + Lb, grad_ref + gb
    assert abs(float(loss.detach()) - L_ref) < 1e-9 * L_ref
    assert rel(sub(gV, lo, hi), sub(grad_ref, lo, hi)) < 1e-9
