"""Write the FP64 oracle's one-step results for the benchmark's extra legs, at sampled nodes.

Calls only the oracle (oracle/) and the seeded generators.  For each leg the benchmark loads
seeded random states into its own grid (in the leg's launch configuration), takes one step and
compares the nodes below with these values:

  * batched 256^3 x 16: members 3 (k = 2 pi) and 12 (k = pi), one step at n = 200 from seeded
    random complex64 states, 64 seeded nodes off the absorbing layers (where the batch's mask,
    set by member 0's energy, is 1 for every member);
  * spinor 384^3 (two spin states, four members): both spinors, one step at n = 300, the 56
    nodes of the full-size spinor parity test (corners, random, inside B's support);
  * auxiliary wave 128^3: one step at n = 17 from seeded random states with the benchmark's
    Gaussian profile on its 512-point axis, 4096 seeded nodes.

    python tests/golden/make_leg_samples.py      # a few minutes on one core

Output: tests/golden/leg_samples_fp64_oracle.npz
"""
import math
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import aux_oracle as ao                  # noqa: E402
from oracle import pstd_oracle as po                 # noqa: E402
from oracle import spinor_oracle as so               # noqa: E402
from paper_2403_04053_gb300 import inputs            # noqa: E402

OUT = os.path.join(HERE, "leg_samples_fp64_oracle.npz")

# the states and nodes the benchmark legs use (bench.py reads these values from the file)
BATCHED = dict(members=(3, 12), seeds=((60, 61), (62, 63)), n=200, nodes=64, node_seed=2420)
SPINOR = dict(seeds=(40, 50), n=300, node_seed=12)
AUX = dict(seeds=(5, 6), n=17, nodes=4096, node_seed=2421, axis=(-16.5, 0.15, 512), sigma=1.0, d0=-4.0)


def spinor_nodes():
    rng = np.random.default_rng(SPINOR["node_seed"])
    nodes = [(0, 0, 0), (383, 383, 383), (5, 200, 379), (192, 192, 192), (150, 240, 145), (239, 145, 200),
             (130, 130, 130), (253, 128, 190)]
    nodes += [tuple(int(v) for v in rng.integers(0, 384, 3)) for _ in range(24)]
    nodes += [tuple(int(v) for v in rng.integers(145, 240, 3)) for _ in range(24)]
    return np.array(nodes)


def main():
    out = {}
    # batched: scalar members through the spinor node evaluator with B = 0 (the up component is
    # the scalar EXACT-form update, pinned in tests/test_oracle_spinor.py)
    wl = inputs.batched_workload()
    sp = wl.spec
    a = sp.abc_cells[0]
    rng = np.random.default_rng(BATCHED["node_seed"])
    nodes = rng.integers(a, sp.n[0] - a, size=(BATCHED["nodes"], 3))
    zero = np.zeros(sp.shape, dtype=np.float32)
    Bz = [zero, zero, zero]
    for b, (s0, s1) in zip(BATCHED["members"], BATCHED["seeds"]):
        inc = wl.incidences[b]
        prev = inputs.random_field_c64(sp.shape, s0)
        cur = inputs.random_field_c64(sp.shape, s1)
        ref = so.step_at_nodes(sp, wl.V, Bz, 0.0, inc.khat, inc.k, inc.ramp_time, (1.0, 0.0),
                               (prev, zero), (cur, zero), BATCHED["n"], nodes)
        out[f"batched_ref_{b}"] = ref[:, 0]
        print(f"batched member {b} done", flush=True)
    out["batched_nodes"] = nodes
    # spinor
    wl = inputs.spinor_workload()
    sp, inc = wl.spec, wl.incidences[0]
    prev = [inputs.random_field_c64(sp.shape, SPINOR["seeds"][0] + b) for b in range(4)]
    cur = [inputs.random_field_c64(sp.shape, SPINOR["seeds"][1] + b) for b in range(4)]
    nodes = spinor_nodes()
    refs = [so.step_at_nodes(sp, wl.V, wl.B, wl.gamma, inc.khat, inc.k, inc.ramp_time, chi,
                             prev[2 * p:2 * p + 2], cur[2 * p:2 * p + 2], SPINOR["n"], [tuple(v) for v in nodes])
            for p, chi in enumerate(wl.chis)]
    out["spinor_ref"] = np.stack(refs)          # [spinor][node][component]
    out["spinor_nodes"] = nodes
    print("spinor done", flush=True)
    # auxiliary wave at 128^3 (whole-array oracle step)
    wl = inputs.gaussian_sum_workload(with_outputs=False)
    sp, inc = wl.spec, wl.incidences[0]
    d_lo, dd, n1 = AUX["axis"]
    d = d_lo + dd * np.arange(n1)
    x = d - AUX["d0"]
    prof = np.exp(-x * x / (4 * AUX["sigma"] ** 2) + 1j * inc.k * x)
    E0 = 0.5 * inc.k ** 2
    sim = po.Simulation(sp, wl.V, inc.khat, inc.k, 0.0, aux=ao.AuxSource1D(d_lo, dd, prof, E0, sp.dt))
    sim.prev = inputs.random_field(sp.shape, AUX["seeds"][0]).astype(np.complex64).astype(np.complex128)
    sim.cur = inputs.random_field(sp.shape, AUX["seeds"][1]).astype(np.complex64).astype(np.complex128)
    sim.n = AUX["n"]
    sim.step(1)
    rng = np.random.default_rng(AUX["node_seed"])
    flat = rng.choice(int(np.prod(sp.shape)), AUX["nodes"], replace=False)
    out["aux_nodes"] = flat
    out["aux_ref"] = sim.cur.ravel()[flat]
    print("aux done", flush=True)
    np.savez_compressed(OUT, **out)
    print(f"wrote {OUT}")


if __name__ == "__main__":
    main()
