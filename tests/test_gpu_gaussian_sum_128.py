"""The benchmarked 128^3 Gaussian-sum pass, in full, against the FP64 oracle (GPU).

The whole pass the benchmark times -- 3000 leapfrog steps with the running DFT over the
last 260, the surface transform to the 256 x 256 Fresnel plane and the 361 x 180 far field
-- run through the C ABI in FP32 (and FP64), compared with the FP64 oracle's results for
the same seeded inputs.  The oracle run takes about 20 minutes on one core, so its results
were written once by tests/golden/make_gaussian_sum_128.py (which calls only the oracle)
as seeded samples: 8192 nodes of the final state, every fourth node of each Huygens plane's
phasors, 48 Fresnel points and 1066 far-field directions.

Tolerances (relative L2 over the samples): FP32 2e-4 on psi and 1e-3 on the plane phasors,
the Fresnel field and the cross-section (the stated FP32 targets); FP64 1e-10.
"""
import os

import numpy as np
import pytest

from paper_2403_04053_gb300 import inputs, pstd

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "gaussian_sum_128_fp64_oracle.npz")


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


@pytest.fixture(scope="module")
def golden():
    return dict(np.load(GOLDEN))


@pytest.fixture(scope="module")
def workload():
    return inputs.gaussian_sum_workload()


@pytest.mark.parametrize("prec,tol_state,tol_out,G", [(pstd.F32, 2e-4, 1e-3, 0), (pstd.F64, 1e-10, 1e-10, 0),
                                                      (pstd.F32, 2e-4, 1e-3, 4)])
def test_full_benchmarked_pass_against_the_fp64_oracle(golden, workload, prec, tol_state, tol_out, G):
    # G = 0: the default cell quadrature; G = 4: the cheaper one, held to the same FP32 targets
    wl = workload
    inc = wl.incidences[0]
    assert int(golden["nsteps"]) == wl.nsteps and tuple(golden["window"]) == (wl.window_first, wl.window_len)
    with pstd.Grid(wl.spec, precision=prec) as g:
        g.set_transform_order(G)
        g.set_potential(wl.V)
        g.set_incidence(0, inc.khat, inc.k, inc.ramp_time)
        g.huygens_dft(0, [0.5 * inc.k ** 2], wl.window_first, wl.window_len)
        g.step(wl.nsteps)
        g.synchronize()
        state = g.get_field(0).ravel()
        phs = g.get_phasors(0, 0)
        psi = g.transform_to_points(0, 0, wl.fresnel_points[golden["fresnel_idx"]])
        ds, f = g.cross_section(0, 0, wl.far_theta[golden["far_idx"]], wl.far_phi[golden["far_idx"]])
    assert rel(state[golden["nodes"]], golden["psi_nodes"]) < tol_state
    assert abs(np.linalg.norm(state) - golden["psi_norm"]) < tol_state * golden["psi_norm"]
    st = int(golden["plane_stride"])
    got_p = np.stack([p[::st, ::st] for p, _ in phs])
    got_d = np.stack([d[::st, ::st] for _, d in phs])
    assert rel(got_p, golden["planes_psi"]) < tol_out and rel(got_d, golden["planes_dpsi"]) < tol_out
    assert rel(psi, golden["fresnel_psi"]) < tol_out
    assert rel(f, golden["far_f"]) < tol_out and rel(ds, golden["far_dsdo"]) < tol_out
