"""Write the FP64 oracle's results for the full 128^3 Gaussian-sum workload.

Calls only the oracle (oracle/) and the seeded workload generator: the whole 3000-step
FP64 run with the running DFT over the last three carrier periods, then the surface
transform at sampled Fresnel-plane points and the far field at sampled directions, as
the benchmark's FP32 pass computes them.  The full state and plane data are too large to
store, so the file keeps seeded samples of each: the GPU test compares its own full run
against them element by element.

    python tests/golden/make_gaussian_sum_128.py      # about 10 minutes on one core

Output: tests/golden/gaussian_sum_128_fp64_oracle.npz
"""
import math
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import ntdf_oracle as no            # noqa: E402
from oracle import pstd_oracle as po            # noqa: E402
from paper_2403_04053_gb300 import inputs       # noqa: E402

OUT = os.path.join(HERE, "gaussian_sum_128_fp64_oracle.npz")
NODE_SAMPLES = 8192
PLANE_STRIDE = 4
FRESNEL_SAMPLES = 48
FAR_STRIDE = 61          # every 61st of the 64980 far-field directions (1066 directions)


def main():
    t0 = time.time()
    wl = inputs.gaussian_sum_workload()
    inc = wl.incidences[0]
    spec = wl.spec
    sim = po.Simulation(spec, wl.V, inc.khat, inc.k, inc.ramp_time, window=(wl.window_first, wl.window_len))
    sim.step(wl.nsteps)
    print(f"steps done in {time.time() - t0:.0f} s", flush=True)
    rng = np.random.default_rng(2412)
    nodes = rng.choice(int(np.prod(spec.shape)), NODE_SAMPLES, replace=False)
    psi_nodes = sim.cur.ravel()[nodes]
    phs = sim.scaled_phasors(0)
    planes_psi = np.stack([p[::PLANE_STRIDE, ::PLANE_STRIDE] for p, _ in phs])
    planes_dpsi = np.stack([d[::PLANE_STRIDE, ::PLANE_STRIDE] for _, d in phs])
    fres_idx = np.sort(rng.choice(len(wl.fresnel_points), FRESNEL_SAMPLES, replace=False))
    fres = no.transform_to_points(spec, inc.k, phs, wl.fresnel_points[fres_idx])
    print(f"transform done in {time.time() - t0:.0f} s", flush=True)
    far_idx = np.arange(0, len(wl.far_theta), FAR_STRIDE)
    ds, f = no.cross_section(spec, inc.k, phs, wl.far_theta[far_idx], wl.far_phi[far_idx])
    np.savez_compressed(OUT, nodes=nodes, psi_nodes=psi_nodes, psi_norm=np.linalg.norm(sim.cur),
                        plane_stride=PLANE_STRIDE, planes_psi=planes_psi, planes_dpsi=planes_dpsi,
                        fresnel_idx=fres_idx, fresnel_psi=fres, far_idx=far_idx, far_f=f, far_dsdo=ds,
                        nsteps=wl.nsteps, window=np.array([wl.window_first, wl.window_len]))
    print(f"wrote {OUT} in {time.time() - t0:.0f} s")


if __name__ == "__main__":
    main()
