"""Benchmark of the PSTD scattering path on GB300.

One step = one pass of the whole hot path over the 128^3 Gaussian-sum workload:
reset, incident-wave tables, 3000 leapfrog steps with the running DFT on the six
virtual planes over the last three carrier periods, the surface transform to the
256 x 256 Fresnel plane and the 361 x 180 far-field cross-section.  FP32 state
(complex64); the FP64 path is run once outside the timed region for the FP32-vs-FP64
comparison.  Inputs are synthetic and seeded (paper_2403_04053_gb300.inputs).

Prints one JSON line (rank 0).  `--impl reference` times the FP64 CPU oracle on a
bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "PSTD cell-updates/s, FP32 vs FP64 at stated error (1 GB300); adjoint/forward time"

# DRAM bytes (read + write) of one cold launch at 128^3: dram__bytes_read.sum +
# dram__bytes_write.sum from an ncu capture of two launches of each kernel (mean); drop an
# entry when its kernel changes
DRAM_TRAFFIC = {"xypass": 33.593e6 + 0.295e6, "zpass": 34.645e6 + 0.0}
# the same for the 256^3 passes of the batched leg (the cluster-fused x+y pass and the z
# pass, steps outside the DFT window), captured with 4 members; the leg scales them by the
# units processed to its own member count
BATCHED_TRAFFIC = {"xypass": 1.0906e9 + 0.9002e9, "zpass": 1.0861e9 + 0.5505e9}
WORKLOAD = "gaussian-sum-128^3"


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


class ClockSampler:
    """nvidia-smi samples of the SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx = float(p[2])
            except ValueError:
                continue
            for name, v in zip(names, p[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def reduce_max(value: float, world: int):
    """Maximum of a per-rank number over all ranks (NCCL on the GPUs, gloo on the host)."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate(t_local: float, world: int, units_per_rank: float):
    """Replicas: every rank processes the same units; the job takes as long as its slowest rank.

    Returns (max-over-ranks seconds per step, whole-job units per second)."""
    t = reduce_max(t_local, world)
    return t, world * units_per_rank / t


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


# ----------------------------------------------------------------------------------
# error against the FP64 oracle
# ----------------------------------------------------------------------------------
ORACLE_SAMPLES = os.path.join(ROOT, "tests", "golden", "gaussian_sum_128_fp64_oracle.npz")


def oracle_error(state, psi, ds, fa):
    """Relative L2 errors of the benchmarked pass's results against the FP64 oracle's results
    for the same seeded 128^3 run, over the stored samples (tests/golden, written by a script
    that runs only the oracle): the final state at 8192 nodes, the Fresnel field at 48 plane
    points and the far field at 1066 directions."""
    try:
        gd = np.load(ORACLE_SAMPLES)
    except OSError:
        return None

    def host(x):
        return x.cpu().numpy() if hasattr(x, "cpu") else np.asarray(x)

    def r(a, b):
        return float(np.linalg.norm(a - b) / np.linalg.norm(b))

    state, psi, ds, fa = host(state).ravel(), host(psi), host(ds), host(fa)
    return {"psi_rel_l2": r(state[gd["nodes"]], gd["psi_nodes"]),
            "fresnel_psi_rel_l2": r(psi[gd["fresnel_idx"]], gd["fresnel_psi"]),
            "f_rel_l2": r(fa[gd["far_idx"]], gd["far_f"]),
            "dsdo_rel_l2": r(ds[gd["far_idx"]], gd["far_dsdo"]),
            "samples": "8192 state nodes, 48 Fresnel points, 1066 far-field directions of the full 3000-step run",
            "targets": {"psi": 2e-4, "cross_sections": 1e-3}}


LEG_SAMPLES = os.path.join(ROOT, "tests", "golden", "leg_samples_fp64_oracle.npz")


def leg_one_step_error(kind, g, wl):
    """One step of a leg's grid, in the leg's launch configuration, from the seeded random states
    for which the FP64 oracle's results at sampled nodes are stored (tests/golden, written by
    make_leg_samples.py, which runs only the oracle); the relative L2 error over those nodes.
    Runs outside the timed regions; it overwrites the grid's state."""
    from paper_2403_04053_gb300 import inputs
    try:
        gd = np.load(LEG_SAMPLES)
    except OSError:
        return None
    shape = wl.spec.shape

    def at(field, nodes):
        return np.array([field[k, j, i] for i, j, k in nodes])

    errs = {}
    if kind == "batched":
        nodes = gd["batched_nodes"]
        for b, (s0, s1) in zip((3, 12), ((60, 61), (62, 63))):
            if b >= g.batch:
                continue
            g.set_field(b, inputs.random_field_c64(shape, s0), inputs.random_field_c64(shape, s1), 200)
        g.step(1)
        for b in (3, 12):
            if b < g.batch:
                ref = gd[f"batched_ref_{b}"]
                errs[f"member_{b}_rel_l2"] = float(np.linalg.norm(at(g.get_field(b), nodes) - ref) / np.linalg.norm(ref))
        errs["sample"] = "one step from seeded random states at n = 200, 64 nodes off the absorbing layers"
    elif kind == "spinor":
        nodes = gd["spinor_nodes"]
        for b in range(4):
            g.set_field(b, inputs.random_field_c64(shape, 40 + b), inputs.random_field_c64(shape, 50 + b), 300)
        g.step(1)
        got = np.stack([np.stack([at(g.get_field(2 * p + s), nodes) for s in range(2)], axis=1) for p in range(2)])
        ref = gd["spinor_ref"]
        errs["rel_l2"] = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
        errs["sample"] = "one step from seeded random states at n = 300, both spinors, 56 nodes (corners, random, B's support)"
    elif kind == "aux":
        flat = gd["aux_nodes"]
        prev = inputs.random_field(shape, 5).astype(np.complex64)
        cur = inputs.random_field(shape, 6).astype(np.complex64)
        g.set_field(0, prev, cur, 17)
        g.step(1)
        ref = gd["aux_ref"]
        errs["rel_l2"] = float(np.linalg.norm(g.get_field(0).ravel()[flat] - ref) / np.linalg.norm(ref))
        errs["sample"] = "one step from seeded random states at n = 17, 4096 seeded nodes"
    errs["target"] = 2e-6
    return errs


# ----------------------------------------------------------------------------------
# roofline of the leapfrog step
# ----------------------------------------------------------------------------------
STEP_KERNELS = ("xpass", "ypass", "zpass", "xypass", "source", "aux")


def step_roofline(kstats, ncell, members, nsteps, t_steps, traffic_per_launch, l2_resident=False):
    """HBM roofline of the whole leapfrog step.

    Algorithmic bytes: one step must read psi^n and psi^{n-1} and write psi^{n+1}, 3 complex64
    = 24 B per cell and member.  `achieved` divides them by the live stepping time per step
    (CUDA events around the steps alone, on the library's stream) and `frac` by the measured
    copy bandwidth.  The step's passes each read psi^n and read-modify-write the partial level
    (24 B a cell per pass); `passes` gives each pass kernel's mean live launch time and its own
    achieved rate on those 24 B, and `traffic_per_step` the DRAM bytes the ncu captures measured
    for the step's launches (null when a kernel changed since its capture)."""
    pk = peaks()
    hbm = pk.get("hbm_gbs", 6800.0)
    alg = 24.0 * ncell * members
    per_step = t_steps / nsteps
    achieved = alg / per_step / 1e9
    passes = {}
    traffic = 0.0
    traffic_known = True
    launches_per_step = 0.0
    for name in STEP_KERNELS:
        n, ms = kstats.get(name, (0, 0.0))
        if not n:
            continue
        launches_per_step += n / nsteps
        if name in ("source", "aux"):
            passes[name] = {"launches": n, "avg_us": round(ms / n * 1e3, 2)}
            continue
        avg = ms / n / 1e3
        passes[name] = {"launches": n, "avg_us": round(avg * 1e6, 2), "achieved_GBs": round(alg / avg / 1e9, 1),
                        "frac": round(alg / avg / 1e9 / hbm, 4)}
        t = traffic_per_launch.get(name)
        if t is None:
            traffic_known = False
        else:
            traffic += t * n / nsteps
    out = {"kernel": "leapfrog step (" + " + ".join(k for k in passes if k not in ("source", "aux")) + ")",
           "bound": "hbm", "achieved": round(achieved, 1), "peak": hbm, "unit": "GB/s", "frac": round(achieved / hbm, 4),
           "traffic": round(traffic) if traffic_known else None,
           "traffic_per_step": round(traffic) if traffic_known else None,
           "traffic_over_algorithmic": round(traffic / alg, 3) if traffic_known else None,
           "algorithmic_bytes_per_step": int(alg), "step_us": round(per_step * 1e6, 2),
           "launches_per_step": round(launches_per_step, 2), "passes": passes,
           "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)" if "hbm_gbs" in pk else "fallback"}
    if l2_resident:
        out["l2_resident"] = True
        out["note"] = ("two levels of the state fit in the 129 MB L2 and stay there between steps: "
                       "an HBM-equivalent rate, not a DRAM measurement")
    return out


# ----------------------------------------------------------------------------------
# GPU arm
# ----------------------------------------------------------------------------------
def run_gpu(args):
    import torch
    from paper_2403_04053_gb300 import inputs, pstd

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    wl = inputs.gaussian_sum_workload(nsteps=args.nsteps)
    spec = wl.spec
    inc = wl.incidences[0]
    w0 = spec.hbar * inc.k ** 2 / (2 * spec.mass)
    ncell = int(np.prod(spec.n))
    stream = torch.cuda.current_stream()
    dev = torch.device("cuda", local)
    V_dev = torch.from_numpy(wl.V).to(dev)
    pts_dev = torch.from_numpy(wl.fresnel_points).to(dev)
    th_dev = torch.from_numpy(wl.far_theta).to(dev)
    ph_dev = torch.from_numpy(wl.far_phi).to(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)   # 256 MB > L2

    def one_pass(g, host=False, step_events=None):
        g.reset()
        g.set_incidence(0, inc.khat, inc.k, inc.ramp_time)
        g.huygens_dft(0, [w0], wl.window_first, wl.window_len)
        if step_events:
            step_events[0].record(stream)
        g.step(wl.nsteps)
        if step_events:
            step_events[1].record(stream)
        if host:
            psi = g.transform_to_points(0, 0, wl.fresnel_points)
            ds, fa = g.cross_section(0, 0, wl.far_theta, wl.far_phi)
        else:
            psi = g.transform_to_points(0, 0, pts_dev)
            ds, fa = g.cross_section(0, 0, th_dev, ph_dev)
        return psi, ds, fa

    g = pstd.Grid(spec, precision=pstd.F32, stream=stream.cuda_stream)
    g.set_potential(V_dev)
    for _ in range(args.warmup):
        one_pass(g)
    torch.cuda.synchronize()
    times, step_times = [], []
    launches0 = g.launch_count()
    barrier(world)
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            flush.fill_(1.0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            se = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
            e0.record(stream)
            psi, ds, fa = one_pass(g, step_events=se)
            e1.record(stream)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1) / 1e3)
            step_times.append(se[0].elapsed_time(se[1]) / 1e3)   # the leapfrog steps of the pass alone
    barrier(world)
    launches = g.launch_count() - launches0
    # per-kernel CUDA-event durations on the library's stream, from one more pass with the
    # library's event timing on (kept out of the timed passes above: the event records
    # cost host time between launches)
    flush.fill_(1.0)
    g.set_timing(True)
    one_pass(g)
    kstats = {name: g.kernel_stats(name) for name in pstd.KERNELS}
    g.set_timing(False)
    # the pass's FP32 results against the FP64 oracle's (stored samples of the same seeded run)
    err_oracle = oracle_error(g.get_field(0), psi, ds, fa)
    t_step, value = aggregate(sum(times) / len(times), world, ncell * wl.nsteps)

    # end to end through host buffers: V, points and angles in, psi and dsigma out
    h2d = wl.V.nbytes + wl.fresnel_points.nbytes + wl.far_theta.nbytes + wl.far_phi.nbytes
    e2e_times = []
    for i in range(0 if args.skip_e2e else max(1, min(3, args.steps))):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        g.set_potential(wl.V)
        psi_h, ds_h, fa_h = one_pass(g, host=True)
        torch.cuda.synchronize()
        e2e_times.append(time.perf_counter() - t0)
    d2h = 0 if args.skip_e2e else psi_h.nbytes + ds_h.nbytes + fa_h.nbytes
    t_e2e, v_e2e = aggregate(sum(e2e_times) / len(e2e_times), world, ncell * wl.nsteps) if e2e_times else (0.0, None)

    roofline = step_roofline(kstats, ncell, 1, wl.nsteps, statistics.median(step_times),
                             DRAM_TRAFFIC, l2_resident=True)
    kernel_ms = {n: {"launches": c, "total_ms": round(t, 3)} for n, (c, t) in kstats.items()}

    # FP64 path once (outside the timed region): throughput and the FP32-vs-FP64 error
    fp64 = None
    if not args.skip_fp64:
        g64 = pstd.Grid(spec, precision=pstd.F64, stream=stream.cuda_stream)
        g64.set_potential(V_dev)
        g64.set_timing(True)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        psi64, ds64, fa64 = one_pass(g64)
        e1.record(stream)
        torch.cuda.synchronize()
        t64 = e0.elapsed_time(e1) / 1e3
        step_ms = sum(g64.kernel_stats(n)[1] for n in ("xpass", "ypass", "zpass", "source"))
        ds32, ds64c = ds.double().cpu().numpy(), ds64.double().cpu().numpy()
        p32, p64 = psi.cpu().numpy(), psi64.cpu().numpy()
        fp64 = {"value": ncell * wl.nsteps / t64, "unit": "cell-updates/s",
                "stepping_only_value": ncell * wl.nsteps / (step_ms / 1e3),
                "fp32_speedup": round(t64 / t_step, 2),
                "err_fp32_vs_fp64": {"dsdo_rel_l2": float(np.linalg.norm(ds32 - ds64c) / np.linalg.norm(ds64c)),
                                     "fresnel_psi_rel_l2": float(np.linalg.norm(p32 - p64) / np.linalg.norm(p64))},
                "err_vs_fp64_oracle": oracle_error(g64.get_field(0), psi64, ds64, fa64)}
        g64.close()
        # the FP64 passes are ALU-bound on GB300: their rate against the measured FP64 FMA peak,
        # on the nominal 5 N log2 N flops of each forward and inverse line FFT (six a cell and
        # step) plus the update's ~30
        f64_peak = pstd.measure_fma_peak(pstd.F64)
        flops_cell = 6 * 5 * math.log2(spec.n[0]) + 30
        ach = flops_cell * fp64["stepping_only_value"] / 1e12
        fp64["roofline"] = {"kernel": "FP64 leapfrog step (x, y, z passes)", "bound": "alu", "achieved": round(ach, 4),
                            "peak": round(f64_peak, 4), "unit": "TFLOP/s", "frac": round(ach / f64_peak, 4),
                            "flops_per_cell_update": flops_cell,
                            "peak_source": "pstd_measure_fma_peak (FP64 FMA chains on every SM, measured here)"}
    g.close()
    fma_peaks = {"fp32_tflops": round(pstd.measure_fma_peak(pstd.F32), 2),
                 "fp64_tflops": round(pstd.measure_fma_peak(pstd.F64), 3),
                 "how": "independent FMA chains, 8 per thread, 8 CTAs of 256 threads per SM, best of 5 launches"}
    # the near transform: (point, cell) pairs per second of the benchmarked pass
    n_tr, ms_tr = kstats["transform"]
    ncells_surface = sum(2 * (spec.huygens_hi[b] - spec.huygens_lo[b]) * (spec.huygens_hi[c] - spec.huygens_lo[c])
                         for (b, c) in ((1, 2), (0, 2), (0, 1)))
    transform = {"points": len(wl.fresnel_points), "surface_cells": ncells_surface, "ms": round(ms_tr, 3),
                 "pairs_per_s": len(wl.fresnel_points) * ncells_surface / (ms_tr / 1e3),
                 "points_per_s": len(wl.fresnel_points) / (ms_tr / 1e3)}

    # adjoint leg: gradient of the Fresnel-plane |Psi| misfit with respect to V on the central
    # 48^3 block (128^3, FP32, 2000 steps, 128^2 points), timed against its forward run
    adjoint = None if args.skip_adjoint else adjoint_leg(pstd, inputs, stream, dev)
    # batched leg: 16 incidences against one potential on a 256^3 grid (HBM-bound regime)
    batched = None if args.skip_batched else batched_leg(pstd, inputs, stream, dev, flush, shell_points=args.shell_points)
    # spinor leg: two spin states of a sigma . B scattering problem on a 384^3 grid
    spinor = None if args.skip_spinor else spinor_leg(pstd, inputs, stream, dev, flush)
    # auxiliary-wave leg: arbitrary incident packets from the 1-D auxiliary axis
    aux = None if args.skip_aux else aux_leg(pstd, inputs, stream, dev, flush)

    out = {
        "metric": METRIC, "value": value, "unit": "cell-updates/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_step * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "c64", "data": "synthetic (seeded Gaussian-sum potential)",
        "config": {"workload": WORKLOAD, "grid": list(spec.n), "time_steps": wl.nsteps, "batch": 1,
                   "dft_window_steps": wl.window_len, "fresnel_points": len(wl.fresnel_points),
                   "far_field_directions": len(wl.far_theta), "parallelism": f"replicas x{world}",
                   "l2": "flushed (256 MB write) between timed steps"},
        "e2e": {"value": v_e2e, "unit": "cell-updates/s", "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h)},
        "roofline": roofline,
        "err_vs_fp64_oracle": err_oracle,
        "fma_peaks": fma_peaks,
        "transform": transform,
        "gpu_launches": int(launches),
        "kernels": kernel_ms,
        "fp64": fp64,
        "adjoint": adjoint,
        "batched": batched,
        "spinor": spinor,
        "aux_source": aux,
    }
    if rank == 0:
        out["clocks"] = clk.summary()
        if not args.skip_cpu:
            out["cpu_baseline"] = cpu_baseline(wl, args.cpu_seconds)
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def batched_leg(pstd, inputs, stream, dev, flush, members=None, nsteps=80, shell_points=1_000_000, force=None):
    """Cell-updates/s of the batched 256^3 x 16 configuration over 80 steps (the last half in
    every member's DFT window), with the step variants chosen by the library's autotuner, the
    HBM roofline of the step, and the surface transform of every member to `shell_points`
    seeded points between 0.5 D^2/lambda and 4 D^2/lambda (one pstd_transform_members call).
    `members` < 16 keeps only the first members (a smaller case of the same kernels); `force`
    (fused_xy, y_pass, z_pass, plans) sets the step variants instead of the autotuner."""
    import torch
    wl = inputs.batched_workload()
    if members:
        wl.incidences = wl.incidences[:members]
    spec = wl.spec
    B = len(wl.incidences)
    g = pstd.Grid(spec, precision=pstd.F32, batch=B, stream=stream.cuda_stream)
    g.set_potential(torch.from_numpy(wl.V).to(dev))
    # each member's DFT window covers the same fraction of the timed steps as its last three
    # carrier periods do of the workload's 3000 (k = 2 pi: 261 steps, k = pi: 1044)
    wins = []
    for b, inc in enumerate(wl.incidences):
        g.set_incidence(b, inc.khat, inc.k, inc.ramp_time)
        wlen = max(1, round(wl.windows[b][1] * nsteps / wl.nsteps))
        wins.append(wlen)
        g.huygens_dft(b, [spec.hbar * inc.k ** 2 / (2 * spec.mass)], nsteps - wlen, wlen)
    ncell = int(np.prod(spec.n))
    if force:
        g.set_variants(*force)
        variants = dict(zip(("fused_xy", "y_pass", "z_pass", "plans"), force), forced=True)
    else:
        variants = g.autotune(6)
    times = []
    for rep in range(3):   # the first repetition is a warm-up
        g.reset()
        flush.fill_(1.0)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        torch.cuda.synchronize()
        ev[0].record(stream)
        g.step(nsteps)
        ev[1].record(stream)
        torch.cuda.synchronize()
        times.append(ev[0].elapsed_time(ev[1]) / 1e3)
    t = statistics.median(times[1:])
    g.reset()
    g.set_timing(True)
    g.step(nsteps)
    ks = {name: g.kernel_stats(name) for name in STEP_KERNELS}
    g.set_timing(False)
    shell = None
    if shell_points:
        D = (spec.tfsf_hi[0] - spec.taper_cells - (spec.tfsf_lo[0] + spec.taper_cells)) * spec.d[0]
        pts = torch.from_numpy(inputs.shell_points(shell_points, 0.5 * D * D, 4.0 * D * D, 2408)).to(dev)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        torch.cuda.synchronize()
        ev[0].record(stream)
        psi = g.transform_members(list(range(B)), [0] * B, pts)
        ev[1].record(stream)
        torch.cuda.synchronize()
        t_tr = ev[0].elapsed_time(ev[1]) / 1e3
        cells = sum(2 * (spec.huygens_hi[b] - spec.huygens_lo[b]) * (spec.huygens_hi[c] - spec.huygens_lo[c])
                    for (b, c) in ((1, 2), (0, 2), (0, 1)))
        shell = {"points": shell_points, "members": B, "surface_cells": cells, "s": round(t_tr, 3),
                 "points_per_s": shell_points * B / t_tr, "pairs_per_s": shell_points * B * cells / t_tr,
                 "geometry": f"radius uniform in [0.5, 4] D^2/lambda, D = {D}, lambda = 1; direction uniform (seed 2408)",
                 "finite": bool(torch.isfinite(psi).all())}
    err = leg_one_step_error("batched", g, wl) if B == 16 else None
    g.close()
    traffic = {k: v * B / 4 for k, v in BATCHED_TRAFFIC.items()}   # captured at 4 members
    return {"workload": f"batched-256^3: {B} incidences (8 Fibonacci directions x k in {{2pi, pi}}) on one "
                        f"Gaussian-sum potential, FP32, {nsteps} steps; DFT windows of the last {max(wins)} (k = pi) "
                        f"and {min(wins)} (k = 2 pi) steps, the workload's 3000-step proportions",
            "value": B * ncell * nsteps / t, "unit": "cell-updates/s", "ms_per_step": t / nsteps * 1e3,
            "state_bytes": 2 * B * ncell * 8,
            "kernels_us": {n: round(v[1] / max(1, v[0]) * 1e3, 1) for n, v in ks.items() if v[0]},
            "variants": variants, "shell_transform": shell, "err_vs_fp64_oracle": err,
            "roofline": step_roofline(ks, ncell, B, nsteps, t, traffic)}


def spinor_leg(pstd, inputs, stream, dev, flush, nsteps=80):
    """Cell-updates/s of the 384^3 spinor configuration (sigma . B of a point dipole, two spin
    states as two spinors = four batch members) over `nsteps` steps, the last half in the DFT
    window; then the 512^2-point Fresnel transform and the 361 x 180 spin-resolved far field of
    every member, each timed with CUDA events."""
    import torch
    wl = inputs.spinor_workload()
    spec = wl.spec
    inc = wl.incidences[0]
    w0 = spec.hbar * inc.k ** 2 / (2 * spec.mass)
    B = 2 * len(wl.chis)
    g = pstd.Grid(spec, precision=pstd.F32, batch=B, stream=stream.cuda_stream)
    g.set_potential(torch.from_numpy(wl.V).to(dev))
    g.set_magnetic_field(wl.B, wl.gamma)
    for p, chi in enumerate(wl.chis):
        g.set_incidence_spinor(p, inc.khat, inc.k, inc.ramp_time, chi)
    # the DFT window covers the same fraction of the timed steps as the workload's last three
    # carrier periods do of its 6000 steps
    wlen = max(1, round(wl.window_len * nsteps / wl.nsteps))
    g.huygens_dft(-1, [w0], nsteps - wlen, wlen)
    ncell = int(np.prod(spec.n))

    def timed(fn):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        torch.cuda.synchronize()
        ev[0].record(stream)
        out = fn()
        ev[1].record(stream)
        torch.cuda.synchronize()
        return ev[0].elapsed_time(ev[1]) / 1e3, out

    times = []
    for rep in range(3):   # the first repetition is a warm-up
        g.reset()
        flush.fill_(1.0)
        times.append(timed(lambda: g.step(nsteps))[0])
    t = statistics.median(times[1:])
    g.reset()
    g.set_timing(True)
    g.step(nsteps)
    ks = {name: g.kernel_stats(name) for name in STEP_KERNELS}
    g.set_timing(False)
    pts = torch.from_numpy(wl.fresnel_points).to(dev)
    th, ph = torch.from_numpy(wl.far_theta).to(dev), torch.from_numpy(wl.far_phi).to(dev)
    t_tr = sum(timed(lambda: g.transform_to_points(b, 0, pts))[0] for b in range(B))
    t_ff = sum(timed(lambda: g.cross_section(b, 0, th, ph))[0] for b in range(B))
    err = leg_one_step_error("spinor", g, wl)
    g.close()
    return {"workload": f"spinor-384^3: gamma sigma . B of a point dipole (cut off inside r = 1 and outside r = 12), "
                        f"unpolarised incidence as 2 spinors = {B} members, FP32, {nsteps} steps "
                        f"({wlen} in the DFT window, the workload's 6000-step proportion)",
            "value": B * ncell * nsteps / t, "unit": "cell-updates/s", "ms_per_step": t / nsteps * 1e3,
            "state_bytes": 2 * B * ncell * 8,
            "kernels_us": {n: round(v[1] / max(1, v[0]) * 1e3, 1) for n, v in ks.items() if v[0]},
            "fresnel_transform_ms": round(t_tr * 1e3, 2), "fresnel_points_per_member": len(wl.fresnel_points),
            "far_field_ms": round(t_ff * 1e3, 2), "far_field_directions": len(wl.far_theta),
            "err_vs_fp64_oracle": err,
            "roofline": step_roofline(ks, ncell, B, nsteps, t, {})}


def aux_leg(pstd, inputs, stream, dev, flush, nsteps=300):
    """The 128^3 Gaussian-sum workload driven by the 1-D auxiliary incident wave (a Gaussian
    profile, sigma = 1, on a 512-point axis) against the same steps with the CW wave: cell-updates/s
    of both, and the per-step cost of evaluating the auxiliary wave on the potential's box."""
    import torch
    wl = inputs.gaussian_sum_workload(with_outputs=False)
    spec, inc = wl.spec, wl.incidences[0]
    w0 = spec.hbar * inc.k ** 2 / (2 * spec.mass)
    # the profile decays to 1e-17 at both ends of the periodic axis (no wrap-around edge)
    d_lo, dd, n1, sigma, d0 = -16.5, 0.15, 512, 1.0, -4.0
    d = d_lo + dd * np.arange(n1)
    x = d - d0
    prof = np.exp(-x * x / (4 * sigma * sigma) + 1j * inc.k * x)
    ncell = int(np.prod(spec.n))
    out = {}
    err_aux = None
    for kind in ("cw", "packet", "aux"):
        g = pstd.Grid(spec, precision=pstd.F32, stream=stream.cuda_stream)
        g.set_potential(torch.from_numpy(wl.V).to(dev))
        if kind == "aux":
            g.set_incidence_aux(0, inc.khat, inc.k, d_lo, dd, prof)
        elif kind == "packet":
            g.set_incidence_packet(0, inc.khat, inc.k, sigma, d0)   # the same packet in closed form
        else:
            g.set_incidence(0, inc.khat, inc.k, inc.ramp_time)
        g.huygens_dft(0, [w0], nsteps - 60, 60)
        times = []
        for rep in range(4):   # the first repetition is a warm-up
            g.reset()
            flush.fill_(1.0)
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
            torch.cuda.synchronize()
            ev[0].record(stream)
            g.step(nsteps)
            ev[1].record(stream)
            torch.cuda.synchronize()
            times.append(ev[0].elapsed_time(ev[1]) / 1e3)
        t = statistics.median(times[1:])
        g.reset()
        g.set_timing(True)
        g.step(nsteps)
        n_aux, ms_aux = g.kernel_stats("aux")
        g.set_timing(False)
        if kind == "aux":
            err_aux = leg_one_step_error("aux", g, wl)
        g.close()
        out[kind] = {"value": ncell * nsteps / t, "ms_per_step": t / nsteps * 1e3}
        if kind == "aux":
            out[kind]["aux_kernel_us_per_step"] = round(ms_aux / nsteps * 1e3, 2)
            out[kind]["aux_launches"] = n_aux
    return {"workload": f"gaussian-sum-128^3, {nsteps} steps (60 in the DFT window), incident wave from the 1-D "
                        f"auxiliary axis ({n1} points, dd = {dd}, Gaussian profile sigma = {sigma}), the same packet "
                        f"in closed form, and the CW wave",
            "unit": "cell-updates/s", "aux": out["aux"], "packet": out["packet"], "cw": out["cw"],
            "err_vs_fp64_oracle": err_aux,
            "aux_overhead": round(out["aux"]["ms_per_step"] / out["cw"]["ms_per_step"] - 1.0, 4),
            "packet_overhead": round(out["packet"]["ms_per_step"] / out["cw"]["ms_per_step"] - 1.0, 4)}


def adjoint_leg(pstd, inputs, stream, dev):
    """Forward run + loss, then the discrete adjoint (transform adjoint + backward sweep with
    sqrt(N) checkpoints), each timed with CUDA events on the library's stream."""
    import torch
    wl, V_target = inputs.adjoint_workload()
    inc = wl.incidences[0]
    w0 = wl.spec.hbar * inc.k ** 2 / (2 * wl.spec.mass)
    lo, hi = (40, 40, 40), (88, 88, 88)
    g = pstd.Grid(wl.spec, precision=pstd.F32, stream=stream.cuda_stream)
    g.set_incidence(0, inc.khat, inc.k, inc.ramp_time)
    g.huygens_dft(0, [w0], wl.window_first, wl.window_len)
    pts = torch.from_numpy(wl.fresnel_points).to(dev)
    g.set_potential(torch.from_numpy(V_target).to(dev))
    g.reset()
    g.step(wl.nsteps)
    target = g.transform_to_points(0, 0, pts).abs()
    V = torch.from_numpy(wl.V).to(dev)
    g.set_potential(V)
    K = math.ceil(math.sqrt(wl.nsteps))
    g.set_checkpointing(K, wl.nsteps)   # the forward run records the backward sweep's checkpoints
    times = []
    for _ in range(3):   # the first repetition is a warm-up
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        torch.cuda.synchronize()
        ev[0].record(stream)
        g.reset()
        g.step(wl.nsteps)
        psi = g.transform_to_points(0, 0, pts)
        ev[1].record(stream)
        mag = psi.abs()
        loss = ((mag - target) ** 2).sum()
        gpts = 2 * (mag - target) * psi / mag
        gph = g.transform_adjoint(0, 0, pts, gpts)
        grad = g.adjoint_gradient(wl.nsteps, gph, lo, hi)
        ev[2].record(stream)
        torch.cuda.synchronize()
        times.append((ev[0].elapsed_time(ev[1]), ev[1].elapsed_time(ev[2])))
    g.close()
    # the same gradient in FP64 (the FP64 path is itself checked against the oracle's discrete
    # adjoint at 48^3 and against central differences at 32 voxels of this workload)
    g64 = pstd.Grid(wl.spec, precision=pstd.F64, stream=stream.cuda_stream)
    g64.set_incidence(0, inc.khat, inc.k, inc.ramp_time)
    g64.huygens_dft(0, [w0], wl.window_first, wl.window_len)
    g64.set_potential(V)
    g64.reset()
    g64.step(wl.nsteps)
    psi64 = g64.transform_to_points(0, 0, pts)
    mag64 = psi64.abs()
    g64pts = 2 * (mag64 - target) * psi64 / mag64
    grad64 = g64.adjoint_gradient(wl.nsteps, g64.transform_adjoint(0, 0, pts, g64pts), lo, hi)
    g64.close()
    grad_err = float(torch.linalg.norm(grad.double() - grad64) / torch.linalg.norm(grad64))
    fwd = statistics.median(t[0] for t in times[1:])
    adj = statistics.median(t[1] for t in times[1:])
    return {"workload": "adjoint-128^3: V on the central 48^3 block (seeded smoothed noise), 2000 steps, "
                        "|Psi| misfit on a 128^2 Fresnel plane", "dtype": "c64",
            "forward_ms": round(fwd, 3), "adjoint_ms": round(adj, 3), "adjoint_over_forward": round(adj / fwd, 3),
            "checkpoint_interval": K, "checkpoints": "recorded by the forward run", "grad_box": [48, 48, 48],
            "loss": float(loss),
            "grad_max_abs": float(grad.abs().max()),
            "err_fp32_vs_fp64_gradient": grad_err,
            "oracle_checks": "FP64 adjoint vs the oracle's discrete adjoint at 48^3 (1e-9) and vs central differences "
                             "at 32 voxels of this workload (1e-6 of max |grad|), tests/test_gpu_adjoint.py"}


# ----------------------------------------------------------------------------------
# CPU oracle (baseline leg and the reference arm)
# ----------------------------------------------------------------------------------
def _oracle_worker(nsteps_total, cmd, barrier, out):
    """One host process: build the 128^3 workload and the FP64 oracle once, then for every
    command (a duration in seconds) wait at the barrier with the other workers and step the
    oracle for that long, putting (steps, elapsed seconds) on `out`; None ends it."""
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    from oracle import pstd_oracle as po
    from paper_2403_04053_gb300 import inputs
    wl = inputs.gaussian_sum_workload(nsteps=nsteps_total, with_outputs=False)
    inc = wl.incidences[0]
    sim = po.Simulation(wl.spec, wl.V, inc.khat, inc.k, inc.ramp_time)
    sim.n = 500
    sim.cur = np.full(wl.spec.shape, 1e-3 + 0j)
    sim.step(1)                         # first-touch of every array outside the timing
    while True:
        seconds = cmd.get()
        if seconds is None:
            break
        barrier.wait()
        t0 = time.perf_counter()
        steps = 0
        while True:
            sim.step(1)
            steps += 1
            if time.perf_counter() - t0 > seconds:
                break
        out.put((steps, time.perf_counter() - t0))


class OraclePool:
    """The FP64 oracle on the host cores: one process per core (started with spawn), each
    stepping its own copy of the 128^3 workload; sample() times all of them together."""

    def __init__(self, nsteps_total: int, workers: int = 0):
        import multiprocessing as mp
        self.workers = workers or (os.cpu_count() or 1)
        ctx = mp.get_context("spawn")
        self.cmd = [ctx.Queue() for _ in range(self.workers)]
        self.out = ctx.Queue()
        self.barrier = ctx.Barrier(self.workers)
        self.procs = [ctx.Process(target=_oracle_worker, args=(nsteps_total, q, self.barrier, self.out))
                      for q in self.cmd]
        for p in self.procs:
            p.start()

    def sample(self, seconds: float):
        """(whole-host cell-updates/s, total steps, wall seconds) over about `seconds`."""
        for q in self.cmd:
            q.put(seconds)
        res = [self.out.get() for _ in self.procs]
        ncell = 128 ** 3
        return sum(ncell * s / t for s, t in res), sum(s for s, _ in res), max(t for _, t in res)

    def close(self):
        for q in self.cmd:
            q.put(None)
        for p in self.procs:
            p.join()


def cpu_baseline(wl, seconds: float):
    pool = OraclePool(wl.nsteps)
    try:
        value, steps, dt = pool.sample(seconds)
    finally:
        pool.close()
    return {"value": value, "unit": "cell-updates/s", "cores": pool.workers, "kind": "oracle",
            "sample": f"{steps} FP64 leapfrog steps of the 128^3 workload in total, {pool.workers} processes (one "
                      f"per host core, numpy FFT) stepping their own copy for {dt:.1f} s"}


def run_reference(args):
    rank, world, local = dist_env()
    if rank != 0:
        return
    from paper_2403_04053_gb300 import inputs
    wl = inputs.gaussian_sum_workload(nsteps=args.nsteps, with_outputs=False)
    per = max(2.0, args.cpu_seconds / 4)
    vals, tot_steps, tot_t = [], 0, 0.0
    pool = OraclePool(args.nsteps)
    workers = pool.workers
    try:
        for i in range(args.warmup + args.steps):
            v, s, t = pool.sample(0.2 if i < args.warmup else per)
            if i >= args.warmup:
                vals.append(v)
                tot_steps += s
                tot_t += t
    finally:
        pool.close()
    value = sum(vals) / len(vals)
    ncell = int(np.prod(wl.spec.n))
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": "cell-updates/s", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": tot_t / args.steps * 1e3,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128",
           "data": "synthetic (seeded Gaussian-sum potential)",
           "config": {"workload": WORKLOAD, "grid": list(wl.spec.n), "sample": "leapfrog steps only, FP64 oracle"},
           "cpu_baseline": {"value": value, "unit": "cell-updates/s", "cores": workers, "kind": "oracle",
                            "sample": f"{tot_steps} FP64 oracle steps of the 128^3 grid over {workers} processes "
                                      f"(one per host core), {args.steps} samples of {per:.1f} s"},
           "e2e": {"value": value, "unit": "cell-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
           "cells_per_step": ncell}
    print(json.dumps(out), flush=True)


def main():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    p.add_argument("--nsteps", type=int, default=3000, help="leapfrog steps per pass (the workload's 3000)")
    p.add_argument("--cpu-seconds", type=float, default=12.0)
    p.add_argument("--skip-cpu", action="store_true")
    p.add_argument("--skip-fp64", action="store_true")
    p.add_argument("--skip-e2e", action="store_true")
    p.add_argument("--skip-adjoint", action="store_true")
    p.add_argument("--skip-batched", action="store_true")
    p.add_argument("--skip-spinor", action="store_true")
    p.add_argument("--skip-aux", action="store_true")
    p.add_argument("--aux-only", action="store_true", help="run only the auxiliary-wave leg and print it")
    p.add_argument("--spinor-only", action="store_true",
                   help="run only the 384^3 spinor leg and print its JSON object (profiling)")
    p.add_argument("--batched-only", action="store_true",
                   help="run only the batched leg (with --batched-members / --batched-steps) and print it")
    p.add_argument("--batched-members", type=int, default=0)
    p.add_argument("--batched-steps", type=int, default=80)
    p.add_argument("--shell-points", type=int, default=1_000_000,
                   help="observation points of the batched leg's shell transform (0 skips it)")
    p.add_argument("--batched-variants", default="",
                   help="fused_xy,y_pass,z_pass,plans for the batched leg instead of the autotuner (profiling)")
    args = p.parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.batched_only:
        import torch
        from paper_2403_04053_gb300 import inputs, pstd
        dev = torch.device("cuda", 0)
        flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
        force = tuple(int(v) for v in args.batched_variants.split(",")) if args.batched_variants else None
        print(json.dumps(batched_leg(pstd, inputs, torch.cuda.current_stream(), dev, flush,
                                     args.batched_members or None, args.batched_steps, args.shell_points, force)),
              flush=True)
    elif args.aux_only:
        import torch
        from paper_2403_04053_gb300 import inputs, pstd
        dev = torch.device("cuda", 0)
        flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
        print(json.dumps(aux_leg(pstd, inputs, torch.cuda.current_stream(), dev, flush)), flush=True)
    elif args.spinor_only:
        import torch
        from paper_2403_04053_gb300 import inputs, pstd
        dev = torch.device("cuda", 0)
        flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
        print(json.dumps(spinor_leg(pstd, inputs, torch.cuda.current_stream(), dev, flush)), flush=True)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
