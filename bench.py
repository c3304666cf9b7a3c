"""Benchmark: Runge-Kutta-Merson steps of the full phase-field model on a 256^3 glass-bead packing.

One "step" = one adaptive Merson attempt on the whole grid: five fused stage kernels
(right-hand side + stage combination), the max-norm error reduction and the device-side
step control (accept/reject, new dt), i.e. one pass of the whole hot path.

Workload (the paper's macro freezing case scaled to a cube): full heat + Allen-Cahn model,
SigmaP1-P reaction, binary64, 256^3 cells of h = 0.3 mm, Boolean bead packing with radii
uniform in [10, 16] voxels to 60% solid, theta = +1 K, top face held at -5 K, other faces
insulated, ice seed in the two top planes, tolerance 1e-6.  Inputs are seeded and synthetic;
the working set (about 2 GB) is far larger than the 129 MB L2, so no flush is needed.

Metric: cell-stage updates per second (cells x 5 right-hand-side evaluations per attempt,
rejected attempts included), summed over ranks.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank runs an independent replica of the workload on its own
GPU (weak scaling; the single-domain solver has no cross-rank exchange).
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

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from paper_2401_01672_gb300 import inputs as I  # noqa: E402

METRIC = "cell-stage updates/s"
UNIT = "cell-stage/s"
SEED = 20240105
N_SIDE = 256
TOL = 1e-6

# Algorithmic work per cell of each Merson stage kernel (full SigmaP1-P model).
# Bytes: stencil input fields + glass field + stage-combination operands read, outputs written,
# each once per cell.  Binary64 path, bytes per cell for stages 1..5:
BYTES_F64 = [56, 72, 88, 104, 104]          # sum 424 = 84.8 B per cell-stage
# Binary32-field form (stage buffers, G and the binary32 copy y32 of the state in 4 B, state y in 8 B;
# stage 1 reads y32 and writes k1 and the increment d2; stages 2-5 read y32 and their increment; stage 5
# reads y and writes y' and its binary32 copy):
BYTES_F32 = [28, 36, 52, 52, 84]            # sum 252 = 50.4 B per cell-stage
# Floating-point operations per cell (FMA = 2, division = 1) of the right-hand side as written
# (blends 6+6+6, fluxes 24, Allen-Cahn 16, latent coupling 6) plus each stage's combination.
FLOPS_RHS = 64
FLOPS_COMB = [4, 6, 8, 12, 24]
# DRAM traffic per cell of the stage-5 kernels from one ncu capture each at 192^3, mid-front state
# (dram__bytes_read.sum + dram__bytes_write.sum over 7,077,888 cells; None once a kernel changes until
# it is captured again).  Binary64: 1072.2 MB -- the method's 104 B plus the per-cell blend
# coefficients (64 B where the Allen-Cahn arithmetic runs, 24 B in the bulk), read instead of
# recomputed on the binary64 pipe that bounds it.  Binary32 form (increments over a binary32 copy of the
# state, which stage 5 writes): 585.6 MB, the method's 84 B.
TRAFFIC_F64_S5_PER_CELL = 151.5
TRAFFIC_F32_S5_PER_CELL = 82.7
KERNEL_BYTES_F64_S5 = None


def shard(items, rank, world):
    """Independent units (instances) of rank `rank` out of `world`: every unit exactly once."""
    return items[rank::world]


def reduce_over_ranks(dist, to_max, to_sum, device):
    """(max over ranks of each value in to_max, sum over ranks of each value in to_sum); the
    values themselves when dist is None (one process)."""
    if dist is None:
        return list(map(float, to_max)), list(map(float, to_sum))
    import torch
    mx = torch.tensor([float(v) for v in to_max], dtype=torch.float64, device=device)
    sm = torch.tensor([float(v) for v in to_sum], dtype=torch.float64, device=device)
    dist.all_reduce(mx, op=dist.ReduceOp.MAX)
    dist.all_reduce(sm, op=dist.ReduceOp.SUM)
    return [float(v) for v in mx.cpu()], [float(v) for v in sm.cpu()]


def env_int(k, d):
    try:
        return int(os.environ.get(k, d))
    except ValueError:
        return d


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def make_workload(kind="full256", n=None):
    """full256: the 256^3 bead packing (radii uniform in [10, 16] voxels); full512: the 512^3 packing
    with lognormal radii (mean 12, log-sd 0.25), freeze then thaw.  n overrides the side (profiling)."""
    if kind == "full512":
        return I.lognormal_case(n or 512)
    n = n or N_SIDE
    return I.full_bead_case(n, SEED, name=f"full_sigmap1p_{n}")


class OracleCrop:
    """The oracle as it stands on a 128 x 128 x 32 crop at the top of the workload (Dirichlet face,
    ice seed, beads).  Setup (the crop's glass field) is not timed."""

    SHAPE = (128, 128, 32)

    def __init__(self, w):
        import oracle
        oracle.build()
        self.oracle = oracle
        c = I.top_crop(w, self.SHAPE, w.params["t_freeze"])
        self.o = oracle.Oracle(c.shape, c.h, c.model, c.reaction, c.params)
        self.G = self.o.glass(c.spheres, c.params["xi_G"])
        self.th, self.ph = c.theta0, c.phi0
        self.n_beads = c.extra["n_spheres"]
        self.cells = int(np.prod(c.shape))
        self.full = w.shape[0]

    def threads(self, n=0):
        return self.oracle.threads(n)

    def step(self):
        self.o.rkm_step(self.G, self.th, self.ph, 0.0, 0.01)

    def describe(self, n, el, threads):
        c = self.SHAPE
        return (f"{n} Merson steps on a {c[0]}x{c[1]}x{c[2]} crop (top of the {self.full}^3 workload, "
                f"{self.n_beads} nearby beads), {threads} thread{'s' if threads > 1 else ''}, {el:.3g} s")


def _time_oracle(oc, seconds, min_steps):
    n, t0 = 0, time.perf_counter()
    while True:
        oc.step()
        n += 1
        el = time.perf_counter() - t0
        if n >= min_steps and el >= seconds:
            return n, el


def cpu_sample(w, seconds=10.0, min_steps=2):
    """cpu_baseline: the oracle timed for about `seconds` on the crop with every host core (OpenMP over
    the loops on cells), and again on one thread."""
    oc = OracleCrop(w)
    full = oc.threads()
    n, el = _time_oracle(oc, seconds, min_steps)
    out = {"value": oc.cells * 5 * n / el, "unit": UNIT, "cores": full, "kind": "oracle",
           "sample": oc.describe(n, el, full)}
    oc.threads(1)
    n1, el1 = _time_oracle(oc, seconds, min_steps)
    oc.threads(full)
    out["single_thread"] = {"value": oc.cells * 5 * n1 / el1, "cores": 1, "sample": oc.describe(n1, el1, 1)}
    return out


def run_reference(args, rank, world):
    """--impl reference: the oracle timed on the host cores (rank 0 only, every core); one step = one
    oracle Merson step on the crop."""
    if rank != 0:
        return
    w = make_workload(args.workload if args.workload in ("full256", "full512") else "full256")
    oc = OracleCrop(w)
    cores = oc.threads()
    for _ in range(args.warmup):
        oc.step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oc.step()
    el = time.perf_counter() - t0
    value = oc.cells * 5 * args.steps / el
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": el * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": w.name, "grid": list(w.shape),
                                            "sample": "128x128x32 crop of the workload",
                                            "l2": "not applicable (CPU)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": oc.describe(args.steps, el, cores)},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def set_tiles(g, tiles):
    """Fixed tile shape, or the autotuner's choice (timed on the grid itself, state unchanged)."""
    if tiles:
        g.set_tiles(*tiles)
    else:
        g.autotune(None)


def timed_window(torch, pf, g, state, steps, warmup, stream, barrier, clk=None):
    """Adaptive attempts from `state` = (theta, phi): `warmup` untimed ones (they also reach the step
    size of the state), then `steps` timed on the device with CUDA events on the grid's stream."""
    g.set_state(state[0], state[1], 0.0, 0.01)
    g.run_to(math.inf, TOL, warmup)
    barrier()
    l0 = pf.pf_kernel_launches()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    if clk:
        clk.__enter__()
    t_wall = time.perf_counter()
    e0.record(stream)
    s = g.run_to(math.inf, TOL, steps)
    e1.record(stream)
    e1.synchronize()
    if clk:
        clk.__exit__(None, None, None)
    t_wall = time.perf_counter() - t_wall
    barrier()
    s["ms"] = e0.elapsed_time(e1)
    s["launches"] = pf.pf_kernel_launches() - l0
    s["wall_s"] = t_wall
    s["attempts"] = s["n_accepted"] + s["n_rejected"]
    return s


def crop_study(pf, w, crop=128, t_freeze=10.0, t_end=20.0):
    """Error of both precision forms against the binary64 oracle (all host cores) on the crop at the
    top centre of the workload, through a freeze-then-thaw cycle: top face -5 K until t_freeze, +2 K
    until t_end, tolerance 1e-6.  Compared at t_freeze (the most ice) and at t_end."""
    import oracle
    oracle.build()
    c = I.top_crop(w, (crop, crop, crop), t_freeze)
    o = oracle.Oracle(c.shape, c.h, c.model, c.reaction, c.params)
    t0 = time.perf_counter()
    G = o.glass(c.spheres, c.params["xi_G"])
    legs = [o.run(G, c.theta0, c.phi0, 0.0, 0.01, t_freeze, TOL, 10 ** 6)]
    legs.append(o.run(G, legs[0]["theta"], legs[0]["phi"], t_freeze, legs[0]["dt"], t_end, TOL, 10 ** 6))
    oracle_s = time.perf_counter() - t0
    ref_u = [o.uwc(G, r["phi"]) for r in legs]
    out = {"crop": [crop] * 3, "beads": c.extra["n_spheres"], "t_freeze": t_freeze, "t_end": t_end,
           "oracle_s": oracle_s, "oracle_threads": oracle.threads(),
           "oracle": [{"attempts": [r["n_accepted"], r["n_rejected"]], "uwc": u["uwc"], "n_ice": u["n_ice"]}
                      for r, u in zip(legs, ref_u)]}
    for prec, key in ((I.PREC_FP64, "f64"), (I.PREC_FP32, "f32_fields")):
        g = pf.Grid(c.shape, c.h, c.model, c.reaction, prec, c.params)
        g.set_geometry(c.spheres)
        g.set_state(c.theta0, c.phi0, 0.0, 0.01)
        rows = []
        for t_stop, ref, ru in zip((t_freeze, t_end), legs, ref_u):
            t0 = time.perf_counter()
            st = g.run_to(t_stop, TOL, 10 ** 6)
            el = time.perf_counter() - t0
            th, ph, _, _ = g.get_state()
            u = g.unfrozen_fraction()
            rows.append({"attempts": [st["n_accepted"], st["n_rejected"]], "wall_s": el,
                         "max_abs_dphi": float(np.max(np.abs(ph - ref["phi"]))),
                         "max_abs_dtheta_K": float(np.max(np.abs(th - ref["theta"]))),
                         "uwc": u["uwc"], "uwc_rel_err": abs(u["uwc"] - ru["uwc"]) / ru["uwc"]})
        g.close()
        out[key] = rows
    return out


def cycle_study(pf, w, stream, tiles, t_freeze=10.0, t_end=20.0):
    """Time to solution of both precision forms on the whole grid through the freeze-then-thaw cycle
    (top face -5 K until t_freeze, +2 K until t_end, tolerance 1e-6): attempts and wall time of each leg,
    the unfrozen water, and the largest phase-field difference between the forms at the end of each leg
    (the oracle cannot run this size; the crop study compares both forms with it)."""
    p = dict(w.params)
    p["t_freeze"] = t_freeze
    out = {"t_freeze": t_freeze, "t_end": t_end}
    ph64 = []
    for prec, key in ((I.PREC_FP64, "f64"), (I.PREC_FP32, "f32_fields")):
        g = pf.Grid(w.shape, w.h, w.model, w.reaction, prec, p, stream=stream)
        g.set_geometry(w.spheres, w.x3_cap)
        g.set_state(w.theta0, w.phi0, 0.0, 0.01)
        g.set_tiles(*tiles[key])
        rows = []
        for leg, t_stop in enumerate((t_freeze, t_end)):
            t0 = time.perf_counter()
            st = g.run_to(t_stop, TOL, 10 ** 6)
            el = time.perf_counter() - t0
            u = g.unfrozen_fraction()
            _, ph, _, _ = g.get_state()
            row = {"attempts": [st["n_accepted"], st["n_rejected"]], "wall_s": el, "uwc": u["uwc"],
                   "n_ice": u["n_ice"]}
            if prec == I.PREC_FP64:
                ph64.append(ph)
            else:
                row["max_abs_dphi_vs_f64"] = float(np.max(np.abs(ph - ph64[leg])))
                row["uwc_rel_vs_f64"] = abs(u["uwc"] - out["f64"][leg]["uwc"]) / out["f64"][leg]["uwc"]
            rows.append(row)
            del ph
        g.close()
        out[key] = rows
    out["time_to_solution_ratio"] = (sum(r["wall_s"] for r in out["f64"]) /
                                     sum(r["wall_s"] for r in out["f32_fields"]))
    return out


def run_sweep(args, rank, world, dist):
    """Time-to-solution of the micro-scale sweep: every instance runs to its equilibrium test
    (ice count unchanged for the time a free front needs to cross 20 cells), its t_end = 4 L/(mu dT) or the attempt cap.
    Under N ranks the instances are sharded (independent problems, no data-path collective); the job's
    time is the slowest rank's, counts are summed."""
    from paper_2401_01672_gb300 import sweep
    inst = I.sweep_instances(args.instances)
    mine = shard(inst, rank, world)
    if dist:
        dist.barrier()
    with ClockSampler(env_int("LOCAL_RANK", 0)) as clk:
        b = sweep.run_batched(mine, max_steps=args.max_steps, keep_phi=True)
    p = sweep.run_plain(mine, max_steps=args.max_steps, keep_phi=True)
    acc = sweep.compare(b, p)
    # the speed-up at the accuracy bars: the instances within the bars, batched again on their own,
    # against their plain binary64 times
    sub = [mine[q] for q in acc["within_bars"]]
    if sub:
        b_sub = sweep.run_batched(sub, max_steps=args.max_steps)
        sub_cmp = {"instances": len(sub), "batched_wall_s": b_sub["wall_s"],
                   "plain_fp64_wall_s": sum(p["instances"][q]["wall_s"] for q in acc["within_bars"])}
        sub_cmp["speedup"] = sub_cmp["plain_fp64_wall_s"] / sub_cmp["batched_wall_s"]
    else:
        sub_cmp = {"instances": 0}
    cells = sum(int(np.prod(i.shape)) for i in mine)
    att_b = sum(r["n_accepted"] + r["n_rejected"] for r in b["instances"])
    att_p = sum(r["n_accepted"] + r["n_rejected"] for r in p["instances"])
    cell_att_b = sum(int(np.prod(i.shape)) * (r["n_accepted"] + r["n_rejected"]) for i, r in zip(mine, b["instances"]))
    eq_b = sum(r["equilibrium"] for r in b["instances"])
    eq_p = sum(r["equilibrium"] for r in p["instances"])
    def nan_low(v):   # a rank with nothing to compare reports NaN: keep it out of the maximum
        return v if v == v else -math.inf

    (wall_b, wall_p, uwc_d, dphi_d), (cells, att_b, att_p, cell_att_b, eq_b, eq_p, n_eq) = reduce_over_ranks(
        dist, [b["wall_s"], p["wall_s"], nan_low(acc["max_uwc_rel_diff"]), nan_low(acc["max_abs_dphi_at_equilibrium"])],
        [cells, att_b, att_p, cell_att_b, eq_b, eq_p, acc["instances_in_equilibrium_both"]], "cuda")
    acc = {"max_uwc_rel_diff": uwc_d if uwc_d > -math.inf else math.nan,
           "max_abs_dphi_at_equilibrium": dphi_d if dphi_d > -math.inf else math.nan,
           "instances_in_equilibrium_both": int(n_eq)}
    if rank == 0:
        line = {"metric": "sweep time-to-solution (equilibrium, t_end or cap)", "value": wall_b, "unit": "s",
                "higher_is_better": False, "n_gpus": world, "steps": args.max_steps, "warmup": 0,
                "dtype": "f32 fields / f64 control", "data": "synthetic", "scaling": "weak",
                "config": {"workload": f"micro_sweep_{len(inst)}", "instances": len(inst), "cells": int(cells),
                           "sizes": [i.shape[0] for i in inst], "cap": args.max_steps, "tol": 1e-6,
                           "instances_per_rank": len(mine)},
                "batched": {"wall_s": wall_b, "attempts": int(att_b), "device_iterations": b["iterations"],
                            "cell_stage_per_s": 5 * cell_att_b / wall_b, "equilibrium": int(eq_b),
                            "tiles_by_zc": b["tiles"][:4]},
                "plain_fp64": {"wall_s": wall_p, "attempts": int(att_p), "equilibrium": int(eq_p)},
                "speedup_vs_plain_fp64": wall_p / wall_b, "accuracy_vs_plain_fp64": acc,
                "within_bars": sub_cmp,
                "clocks": clk.summary()}
        print(json.dumps(line), flush=True)


# The paper's Table 3: wall-clock of its whole macro runs (10 h of physical time) on CPU nodes with
# two 16-core AMD EPYC 7281 each (hybrid MPI/OpenMP), hours:minutes -> seconds.
PAPER_TABLE3 = {
    100: {"cores": 32, "sigmap1p_large": 71 * 60, "sigmap1p_small": 75 * 60, "gradp_large": 162 * 60,
          "temp_gamma2": 23 * 60},
    200: {"cores": 128, "sigmap1p_large": 549 * 60, "sigmap1p_small": 520 * 60, "gradp_large": 613 * 60,
          "temp_gamma2": 566 * 60},
    400: {"cores": 384, "sigmap1p_small": 5431 * 60, "temp_gamma2": 4457 * 60},
}
MACRO_CASES = {
    "sigmap1p_large": (I.MODEL_FULL, I.REACT_SIGMAP1P, "large", 2.0),
    "sigmap1p_small": (I.MODEL_FULL, I.REACT_SIGMAP1P, "small", 2.0),
    "sigmap1p_tiny": (I.MODEL_FULL, I.REACT_SIGMAP1P, "tiny", 2.0),
    "gradp_large": (I.MODEL_FULL, I.REACT_GRADP, "large", 2.0),
    "gradp_small": (I.MODEL_FULL, I.REACT_GRADP, "small", 2.0),
    "temp_gamma2": (I.MODEL_TEMP, I.REACT_SIGMAP1P, "large", 2.0),
    "temp_gamma10": (I.MODEL_TEMP, I.REACT_SIGMAP1P, "large", 10.0),
}


def run_macro(args, rank, world):
    """The paper's macro-scale parametric study (Sec. 3.1-3.2) on the vessel at N3 cells: 5 h cooling
    through the cap at -25 K, 5 h heating at +20 K, binary64 (or the binary32-field form with --form f32),
    tol 1e-6.  Reports each run's wall time
    next to the paper's Table 3 (its CPU cluster; context) and the qualitative findings the paper
    states about the ice-fraction curves.  Rank 0 only (one run = one GPU)."""
    if rank != 0:
        return
    from paper_2401_01672_gb300 import macro, pf
    names = list(MACRO_CASES) if args.macro_cases == "all" else args.macro_cases.split(",")
    runs = {}
    with ClockSampler(env_int("LOCAL_RANK", 0)) as clk:
        for nm in names:
            model, rx, sigma, gamma = MACRO_CASES[nm]
            w = I.macro_case(args.macro_n3, model, rx, sigma=sigma, gamma=gamma)
            runs[nm] = macro.run_case(w, max_attempts=args.macro_cap,
                                      precision=I.PREC_FP32 if args.form == "f32" else I.PREC_FP64)
            print(json.dumps({"case": nm, "status": runs[nm]["status"], "wall_s": runs[nm]["wall_s"],
                              "attempts": runs[nm]["attempts"]}), file=sys.stderr, flush=True)
    # water above the bead bed, as a share of all water: the ice fraction at which a front coming down
    # from the cap reaches the bed
    w0 = I.macro_case(args.macro_n3, I.MODEL_FULL)
    g = pf.Grid(w0.shape, w0.h, w0.model, w0.reaction, I.PREC_FP64, w0.params)
    g.set_geometry(w0.spheres, w0.x3_cap)
    G = g.get_glass().reshape(w0.shape[2], -1)
    g.close()
    z = (np.arange(w0.shape[2]) + 0.5) * w0.h
    water = G < 0.5
    above = float(water[z > w0.extra["bed_top"]].sum() / water.sum())
    summ = {nm: macro.summary(r) for nm, r in runs.items()}

    def dist(a, b):
        return macro.curve_distance(runs[a], runs[b]) if a in runs and b in runs else None

    def early(a, b):   # largest difference while both fronts, coming down from the cap, are above the bed
        if a not in runs or b not in runs:
            return None

        def cooling_above(r):
            return {round(p["t"], 6): p["ice_fraction"] for p in r["curve"]
                    if p["t"] <= I.MACRO_T_FREEZE and p["ice_fraction"] < above}
        ca, cb = cooling_above(runs[a]), cooling_above(runs[b])
        d = [abs(v - cb[t]) for t, v in ca.items() if t in cb]
        return max(d) if d else None

    def tf(nm, key):
        return summ[nm][key] if nm in summ else None

    checks = {
        "models_agree_before_bed (max |diff| while the front is above the bed)":
            {"sigmap1p_small_vs_temp": early("sigmap1p_small", "temp_gamma2"),
             "sigmap1p_large_vs_temp": early("sigmap1p_large", "temp_gamma2")},
        "large_sigma_freezes_later (t_half_freeze large >= small >= tiny)":
            [tf("sigmap1p_large", "t_half_freeze_s"), tf("sigmap1p_small", "t_half_freeze_s"),
             tf("sigmap1p_tiny", "t_half_freeze_s")],
        "large_sigma_thaws_earlier (t_half_thaw large <= small <= tiny)":
            [tf("sigmap1p_large", "t_half_thaw_s"), tf("sigmap1p_small", "t_half_thaw_s"),
             tf("sigmap1p_tiny", "t_half_thaw_s")],
        "sigmap1p_approaches_temp_as_sigma_decreases (max |diff| to Temp: large, small, tiny)":
            [dist("sigmap1p_large", "temp_gamma2"), dist("sigmap1p_small", "temp_gamma2"),
             dist("sigmap1p_tiny", "temp_gamma2")],
        "temp_gamma_insensitive (max |diff| gamma 2 vs 10)": dist("temp_gamma2", "temp_gamma10"),
        "gradp (status, max phi)": {nm: [runs[nm]["status"], summ[nm]["phi_max"]]
                                    for nm in runs if nm.startswith("gradp")},
    }
    paper = PAPER_TABLE3.get(args.macro_n3, {})
    headline = "sigmap1p_small" if "sigmap1p_small" in runs else names[0]
    line = {"metric": "macro freeze-thaw run wall time (10 h physical)", "value": runs[headline]["wall_s"],
            "unit": "s", "higher_is_better": False, "n_gpus": 1, "steps": runs[headline]["attempts"], "warmup": 0,
            "dtype": "f32 fields / f64 state" if args.form == "f32" else "f64", "data": "synthetic",
            "scaling": "weak",
            "config": {"workload": f"macro_vessel_n3_{args.macro_n3}", "grid": list(w0.shape), "h_m": w0.h,
                       "beads": w0.extra["n_spheres"], "bed_top_m": w0.extra["bed_top"], "tol": 1e-6,
                       "headline_case": headline},
            "runs": {nm: {k: r[k] for k in ("status", "wall_s", "attempts", "accepted", "cells", "tiles_by_zc")}
                     | {"cell_stage_per_s": 5 * r["cells"] * r["attempts"] / r["wall_s"] if r["wall_s"] else None}
                     | summ[nm] for nm, r in runs.items()},
            "paper_table3_s": paper, "water_above_bed_fraction": above, "qualitative_checks": checks,
            "curves": {nm: [[round(p["t"], 3), round(p["ice_fraction"], 5)] for p in r["curve"]]
                       for nm, r in runs.items()},
            "clocks": clk.summary()}
    print(json.dumps(line), flush=True)


def run_uwc(args, rank, world):
    """Micro-scale unfrozen water content against supercooling (Sec. 3.3) on an ordered (fcc-like) and a
    random (settled) bead structure of radius 5 um: every (structure, dT) instance in one batched
    binary32 run to its equilibrium test; UWC over the bottom half of the vessel.  The paper compares
    its curves with measurements that are not available here; the bench reports the curves and the two
    trends the paper states: UWC falls as the supercooling grows, and the structure with the larger void
    fraction holds less unfrozen water.  Rank 0 only."""
    if rank != 0:
        return
    from paper_2401_01672_gb300 import sweep
    inst = I.uwc_instances(n3=args.uwc_n3)
    with ClockSampler(env_int("LOCAL_RANK", 0)) as clk:
        b = sweep.run_batched(inst, max_steps=args.max_steps)
    curves, void = {}, {}
    for i, r in zip(inst, b["instances"]):
        curves.setdefault(i.label, []).append({"dT": i.dT, "uwc_percent": 100.0 * r["uwc"],
                                               "equilibrium": bool(r["equilibrium"]), "t": r["t"],
                                               "attempts": r["n_accepted"] + r["n_rejected"]})
        if i.label not in void:
            m = I.sharp_solid_mask(i.shape, i.spheres / i.h)[: i.shape[2] // 2]
            void[i.label] = float(1.0 - m.mean())
    # UWC falls with the supercooling and levels off at a few tenths of a percent at the largest ones;
    # differences below FLOOR_TIE percentage points count as ties
    FLOOR_TIE = 0.25
    mono = {k: all(a["uwc_percent"] >= c["uwc_percent"] - FLOOR_TIE for a, c in zip(v, v[1:]))
            for k, v in curves.items()}
    labels = sorted(void, key=lambda k: void[k])   # denser structure first
    order = None
    if len(labels) == 2:
        lo_void, hi_void = curves[labels[0]], curves[labels[1]]
        order = all(h["uwc_percent"] <= l["uwc_percent"] for l, h in zip(lo_void, hi_void))
    line = {"metric": "micro-scale UWC vs supercooling, batched time-to-equilibrium", "value": b["wall_s"], "unit": "s",
            "higher_is_better": False, "n_gpus": 1, "steps": args.max_steps, "warmup": 0,
            "dtype": "f32 fields / f64 control", "data": "synthetic", "scaling": "weak",
            "config": {"workload": f"uwc_vs_dT_n3_{args.uwc_n3}", "instances": len(inst), "grid": list(inst[0].shape),
                       "bead_radius_m": float(inst[0].spheres[0, 3]), "region": "bottom half",
                       "void_fraction_bottom_half": void},
            "batched": {"wall_s": b["wall_s"], "device_iterations": b["iterations"], "tiles_by_zc": b["tiles"][:2]},
            "curves": curves,
            "checks": {"uwc_falls_with_supercooling (ties below 0.25 points)": mono,
                       "larger_void_holds_less_unfrozen_water": order},
            "clocks": clk.summary()}
    print(json.dumps(line), flush=True)


# Layers of the warm-start network timed by --workload conv: (label, samples, side, cin, cout); the first
# four are the 256^3 inference levels, the last two the 64^3 training batches at the widest levels.
CONV_LAYERS = [("infer_l0_256", 1, 256, 16, 16), ("infer_l1_128", 1, 128, 32, 32), ("infer_l2_64", 1, 64, 64, 64),
               ("infer_l3_32", 1, 32, 128, 128), ("train_l2_32x8", 8, 32, 128, 64), ("train_l0_64x8", 8, 64, 32, 16)]


def run_conv(args, rank, world):
    """Forward 3x3x3 convolutions of the warm-start network on the tensor cores (tcgen05, TMA operands,
    TMEM accumulators), bf16 in and out, fp32 accumulation: device time per layer with CUDA events on
    the launching stream, TFLOP/s (2 x 27 x cin x cout flops per voxel) against the measured bf16 dense
    peak.  Inputs of the larger layers exceed L2.  Rank 0 only."""
    if rank != 0:
        return
    import torch
    from paper_2401_01672_gb300 import nn
    L = nn._lib()
    peaks, kind = load_peaks()
    stream = torch.cuda.Stream()
    g = torch.Generator(device="cuda").manual_seed(SEED)
    out = {}
    with ClockSampler(env_int("LOCAL_RANK", 0)) as clk, torch.cuda.stream(stream):
        for (label, n, side, cin, cout) in CONV_LAYERS:
            nv = n * side ** 3
            x = torch.randn((nv, cin), device="cuda", generator=g).to(torch.bfloat16)
            w = (torch.randn((27, cout, cin), device="cuda", generator=g) * 0.05).to(torch.bfloat16)
            b = torch.zeros(cout, device="cuda")
            y = torch.empty((nv, cout), device="cuda", dtype=torch.bfloat16)
            a = (nn._p(x), cin, 0, nn._p(w), cin, cout, nn._p(b), 1, 0, nn._p(y), None, cout, 0, 0, n, side, side, side,
                 C_void(stream.cuda_stream))
            for _ in range(max(3, args.warmup)):
                nn._ck(L.pfnn_conv3d(*a), label)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            reps = max(5, args.steps)
            e0.record(stream)
            for _ in range(reps):
                L.pfnn_conv3d(*a)
            e1.record(stream)
            e1.synchronize()
            ms = e0.elapsed_time(e1) / reps
            tf = 2.0 * 27 * cin * cout * nv / (ms * 1e-3) / 1e12
            io_gbs = nv * (cin + cout) * 2 / (ms * 1e-3) / 1e9
            halo = cin in (16, 32) and cout in (16, 32) and side >= 16
            out[label] = {"samples": n, "side": side, "cin": cin, "cout": cout, "ms": ms, "tflops": tf,
                          "frac_of_bf16_peak": tf / peaks["bf16_tflops"],
                          "kernel": "k_conv_halo" if halo else "k_conv_umma",
                          "io_gbs": io_gbs, "frac_of_hbm": io_gbs / peaks["hbm_gbs"]}
        nn.check_device()
    top = max(out, key=lambda k: out[k]["tflops"])
    line = {"metric": "warm-start 3x3x3 convolution throughput (forward, tcgen05)", "value": out[top]["tflops"],
            "unit": "TFLOP/s", "higher_is_better": True, "n_gpus": 1, "steps": max(5, args.steps),
            "warmup": max(3, args.warmup), "dtype": "bf16 (fp32 accumulation)", "data": "synthetic", "scaling": "weak",
            "config": {"workload": "warmstart_conv_layers", "best_layer": top},
            "roofline": {"bound": "tensor", "kernel": "k_conv_umma", "achieved": out[top]["tflops"],
                         "peak": peaks["bf16_tflops"], "unit": "TFLOP/s",
                         "frac": out[top]["tflops"] / peaks["bf16_tflops"], "peak_source": kind, "traffic": None},
            "layers": out, "clocks": clk.summary()}
    # the narrow layer is bound by memory traffic, not by the tensor cores: its input and output bytes
    # against the copy bandwidth
    nl = out.get("infer_l0_256")
    if nl:
        line["roofline_narrow"] = {"bound": "hbm", "kernel": nl["kernel"], "layer": "infer_l0_256",
                                   "achieved": nl["io_gbs"], "peak": peaks["hbm_gbs"], "unit": "GB/s",
                                   "frac": nl["frac_of_hbm"], "peak_source": kind, "traffic": None}
    print(json.dumps(line), flush=True)


def C_void(v):
    import ctypes
    return ctypes.c_void_p(v)


def run_warmstart(args, rank, world):
    """Learned warm start: equilibria of 64^3 instances from the batched solver -> BF16 encoder-decoder
    trained with the library's kernels -> inference on larger packings -> binary64 RKM relaxation to the
    equilibrium test, against the plain binary64 run from the nucleation seed."""
    import torch
    from paper_2401_01672_gb300 import warmstart as WS
    if rank != 0:
        return
    t0 = time.perf_counter()
    train = I.warmstart_instances(args.train_samples, 64, seed=20240109)
    t_gen0 = time.perf_counter()
    G, feat, P, stats = WS.generate(train)
    torch.cuda.synchronize()
    t_gen = time.perf_counter() - t_gen0
    t_tr0 = time.perf_counter()
    net, hist = WS.train(G, feat, P, steps=args.train_steps, batch=4, log_every=max(1, args.train_steps // 10))
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t_tr0
    tests = I.warmstart_instances(args.tests, args.test_side, seed=20240110)
    rows = []
    for inst in tests:
        cold, phi_c, w_c, Gt = WS.relax(inst, inst.phi0)
        torch.cuda.synchronize()
        ti = time.perf_counter()
        phi_pred = WS.predict(net, inst, Gt)
        torch.cuda.synchronize()
        t_inf = time.perf_counter() - ti
        warm, phi_w, w_w, _ = WS.relax(inst, phi_pred)
        rows.append({"dT": inst.dT, "sigma_scale": inst.sigma_scale,
                     "cold": {"attempts": cold["n_accepted"] + cold["n_rejected"], "wall_s": w_c,
                              "equilibrium": cold["equilibrium"], "t_eq": cold["t_eq"], "uwc": cold["uwc"]},
                     "warm": {"attempts": warm["n_accepted"] + warm["n_rejected"], "wall_s": w_w + t_inf,
                              "inference_s": t_inf, "equilibrium": warm["equilibrium"], "t_eq": warm["t_eq"],
                              "uwc": warm["uwc"]},
                     "max_abs_dphi_warm_vs_cold": float(np.max(np.abs(phi_w - phi_c))),
                     "max_abs_dphi_pore_bulk": float(np.max(np.abs(phi_w - phi_c)[
                         (1.0 - inst.params["zeta"] * Gt) > 0.5])),
                     "cells_off_by_1e-3": float(np.mean(np.abs(phi_w - phi_c) > 1e-3)),
                     "max_abs_dphi_prediction_vs_cold": float(np.max(np.abs(phi_pred - phi_c))),
                     "uwc_rel_diff": abs(warm["uwc"] - cold["uwc"]) / max(abs(cold["uwc"]), 1e-12)})
    from paper_2401_01672_gb300 import sweep as SW
    for r in rows:
        r["within_bars"] = bool(r["cold"]["equilibrium"] and r["warm"]["equilibrium"] and
                                r["max_abs_dphi_warm_vs_cold"] <= SW.BAR_DPHI and r["uwc_rel_diff"] <= SW.BAR_UWC_REL)
    # the speed-up counts only the instances whose warm-started result meets the accuracy bars
    good = [r for r in rows if r["within_bars"]]
    cold_s = sum(r["cold"]["wall_s"] for r in good)
    warm_s = sum(r["warm"]["wall_s"] for r in good)
    line = {"metric": "time-to-equilibrium, learned warm start + binary64 relaxation vs plain binary64",
            "value": warm_s if good else None, "unit": "s", "higher_is_better": False, "n_gpus": world,
            "steps": args.train_steps,
            "instances_within_bars": f"{len(good)} of {len(rows)} (max|dphi| <= {SW.BAR_DPHI}, "
                                     f"UWC within {SW.BAR_UWC_REL:.1%} relative, both in equilibrium)",
            "all_instances": {"plain_fp64_s": sum(r["cold"]["wall_s"] for r in rows),
                              "warm_s": sum(r["warm"]["wall_s"] for r in rows)},
            "warmup": 0, "dtype": "bf16 network (fp32 accumulation), f64 relaxation", "data": "synthetic",
            "scaling": "weak",
            "config": {"workload": f"warmstart_64_to_{args.test_side}", "train_samples": args.train_samples,
                       "train_steps": args.train_steps, "test_side": args.test_side, "tests": args.tests},
            "plain_fp64_s": cold_s, "speedup_vs_plain_fp64": cold_s / warm_s if good and warm_s > 0 else None,
            "data_generation_s": t_gen, "train_s": t_train,
            "train_equilibria": sum(1 for r in stats if r["equilibrium"]), "loss_history": hist, "tests": rows,
            "wall_total_s": time.perf_counter() - t0}
    print(json.dumps(line), flush=True)


def run_stages(args, rank, world):
    """Stage kernels only, for profiler captures: the bead workload at --size (default 192) from its
    mid-front state, one precision form (--form), the tile shape given (--tiles, default 4 x 12) or the
    autotuner's, one attempt of warm-up then --steps attempts launched one kernel at a time
    (pf_profile_stages: stages 1..5 then the controller per attempt).  Prints the stage times."""
    import torch
    from paper_2401_01672_gb300 import pf
    if rank != 0:
        return
    w = make_workload("full256", args.size or 192)
    prec = I.PREC_FP32 if args.form == "f32" else I.PREC_FP64
    g = pf.Grid(w.shape, w.h, w.model, w.reaction, prec, w.params)
    g.set_geometry(w.spheres, w.x3_cap)
    mid = I.midfront_state(w, g.get_glass())
    g.set_state(mid[0], mid[1], 0.0, 0.01)
    set_tiles(g, args.tiles or (4, 12))
    g.profile_stages(1)
    prof = g.profile_stages(args.steps)
    torch.cuda.synchronize()
    print(json.dumps({"workload": f"stages_{args.form}_{w.shape[0]}", "tiles_by_zc": list(g.get_tiles()),
                      "attempts": args.steps, "stage_ms": prof}), flush=True)
    g.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp32-form", action="store_true")
    ap.add_argument("--tiles", type=int, nargs=2, metavar=("BY", "ZC"), default=None,
                    help="fixed tile shape (block height, z chunk) instead of the autotuner's choice")
    ap.add_argument("--workload", default="full256",
                    choices=["full256", "full512", "sweep48", "warmstart", "macro", "uwc", "conv", "stages"],
                    help="full256: the binary64 bead workload (default); full512: the 512^3 lognormal packing, both "
                         "forms, with the crop error study; sweep48: the 48-instance micro-scale "
                         "sweep, batched binary32 persistent run vs the plain binary64 method")
    ap.add_argument("--no-crop-study", action="store_true", help="full512: skip the 128^3 crop error study")
    ap.add_argument("--no-cycle", action="store_true",
                    help="full512: skip the whole-grid freeze-then-thaw cycle of both forms (time to solution)")
    ap.add_argument("--form", default="f64", choices=["f64", "f32"], help="stages, macro: precision form")
    ap.add_argument("--max-steps", type=int, default=600, help="sweep48, uwc: attempt cap per instance")
    ap.add_argument("--macro-n3", type=int, default=100, help="macro: cells along the vessel height (100/200/400)")
    ap.add_argument("--macro-cap", type=int, default=1_500_000, help="macro: attempt cap per run")
    ap.add_argument("--uwc-n3", type=int, default=120, help="uwc: cells along the vessel height")
    ap.add_argument("--macro-cases", default="all",
                    help="macro: comma-separated subset of sigmap1p_large,sigmap1p_small,sigmap1p_tiny,"
                         "gradp_large,gradp_small,temp_gamma2,temp_gamma10")
    ap.add_argument("--instances", type=int, default=48, help="sweep48: number of instances")
    ap.add_argument("--train-samples", type=int, default=2000, help="warmstart: 64^3 training equilibria")
    ap.add_argument("--train-steps", type=int, default=1500, help="warmstart: Adam steps")
    ap.add_argument("--test-side", type=int, default=256, help="warmstart: side of the inference grids")
    ap.add_argument("--tests", type=int, default=2, help="warmstart: number of inference instances")
    ap.add_argument("--size", type=int, default=None, help="grid side (default: the workload's; "
                    "smaller sizes are for profiling captures only)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3

    world = env_int("WORLD_SIZE", 1)
    rank = env_int("RANK", 0)
    local = env_int("LOCAL_RANK", 0)

    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2401_01672_gb300 import pf

    torch.cuda.set_device(local)
    if args.workload == "warmstart":
        run_warmstart(args, rank, world)
        return
    if args.workload == "macro":
        run_macro(args, rank, world)
        return
    if args.workload == "uwc":
        run_uwc(args, rank, world)
        return
    if args.workload == "conv":
        run_conv(args, rank, world)
        return
    if args.workload == "stages":
        run_stages(args, rank, world)
        return
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if args.workload == "sweep48":
        run_sweep(args, rank, world, dist)
        if dist:
            dist.destroy_process_group()
        return

    w = make_workload(args.workload, args.size)
    stream = torch.cuda.Stream()
    peaks, peak_kind = load_peaks()

    def barrier():
        if dist:
            dist.barrier()
        torch.cuda.synchronize()

    # ---------------- binary64: the mid-front window (headline) and the window after t = 0
    g = pf.Grid(w.shape, w.h, w.model, w.reaction, I.PREC_FP64, w.params, stream=stream)
    g.set_geometry(w.spheres, w.x3_cap)
    G_host = g.get_glass()
    mid = I.midfront_state(w, G_host)
    t0_state = (w.theta0, w.phi0)
    g.set_state(mid[0], mid[1], 0.0, 0.01)
    set_tiles(g, args.tiles)
    tiles = g.get_tiles()
    clk = ClockSampler(local)
    s = timed_window(torch, pf, g, mid, args.steps, args.warmup, stream, barrier, clk)
    prof = g.profile_stages(3)                        # dominant kernel, timed live on the grid's stream
    s0 = timed_window(torch, pf, g, t0_state, args.steps, args.warmup, stream, barrier)
    prof0 = g.profile_stages(3)
    ms, launches, attempts, t_wall = s["ms"], s["launches"], s["attempts"], s["wall_s"]
    local_units = w.n_cells * 5 * attempts
    (ms_max,), (units,) = reduce_over_ranks(dist, [ms], [local_units], "cuda")
    value = units / (ms_max * 1e-3)
    windows = {"midfront": {"value": value, "ms_per_step": ms / max(attempts, 1), "attempts": attempts,
                            "accepted": s["n_accepted"]},
               "t0": {"value": w.n_cells * 5 * s0["attempts"] / (s0["ms"] * 1e-3),
                      "ms_per_step": s0["ms"] / max(s0["attempts"], 1), "attempts": s0["attempts"],
                      "accepted": s0["n_accepted"],
                      "stage_ms": dict(zip(["stage1", "stage2", "stage3", "stage4", "stage5", "controller"], prof0))}}

    stage_names = ["stage1", "stage2", "stage3", "stage4", "stage5", "controller"]
    top = int(np.argmax(prof[:5]))
    top_ms = prof[top]
    flops = (FLOPS_RHS + FLOPS_COMB[top]) * w.n_cells
    fp64_meas, fp32_meas, copy_meas = pf.pf_measure_peaks()
    fp64_peak_tflops = 152 * 2 * 2 * 2.07e9 / 1e12   # 152 SMs x 2 binary64 FMA/clk x 2 flop x 2.07 GHz
    achieved_tf = flops / (top_ms * 1e-3) / 1e12
    roofline = {"bound": "alu", "kernel": f"merson_{stage_names[top]}_full_sigmap1p_f64",
                "achieved": achieved_tf, "peak": fp64_peak_tflops, "unit": "TFLOP/s",
                "frac": achieved_tf / fp64_peak_tflops,
                "traffic": (TRAFFIC_F64_S5_PER_CELL * w.n_cells if (top == 4 and TRAFFIC_F64_S5_PER_CELL) else None),
                "peak_measured_fp64_tflops": fp64_meas, "frac_of_measured": achieved_tf / fp64_meas,
                "measured_fp32_tflops": fp32_meas, "measured_copy_gbs": copy_meas,
                "algorithmic_per_launch": {"flops": flops, "bytes": BYTES_F64[top] * w.n_cells},
                "kernel_bytes_per_launch": (KERNEL_BYTES_F64_S5 * w.n_cells if (top == 4 and KERNEL_BYTES_F64_S5) else None),
                "peak_source": "derived: 152 SMs x 2 FP64 FMA/clk x 2 flop x 2.07 GHz (binary64 pipe)",
                "hbm_achieved_gbs": BYTES_F64[top] * w.n_cells / (top_ms * 1e-3) / 1e9,
                "hbm_peak_gbs": peaks["hbm_gbs"], "hbm_peak_source": peak_kind,
                "stage_ms": dict(zip(stage_names, prof))}

    # ---------------- e2e: host-resident state in pinned memory, copies inside the timed region
    pin_th = torch.from_numpy(mid[0].copy()).pin_memory()
    pin_ph = torch.from_numpy(mid[1].copy()).pin_memory()
    barrier()
    e2e_steps = max(3, args.steps // 2)
    t0 = time.perf_counter()
    e2e_attempts = 0
    for _ in range(e2e_steps):
        g.set_state(pin_th, pin_ph, 0.0, s["dt"])
        r = g.run_to(math.inf, TOL, 1)
        e2e_attempts += r["n_accepted"] + r["n_rejected"]
        u = g.unfrozen_fraction()
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e = {"value": w.n_cells * 5 * e2e_attempts / e2e_s * (units / local_units), "unit": UNIT,
           "h2d_bytes_per_step": 2 * 8 * w.n_cells, "d2h_bytes_per_step": 2 * 136 + 32,
           "note": "per step: pf_set_state from pinned host theta/phi, one pf_run_to attempt, pf_unfrozen_fraction"}
    g.close()

    # ---------------- binary32-field form on the same workload and windows
    forms = {}
    if not args.no_fp32_form:
        g32 = pf.Grid(w.shape, w.h, w.model, w.reaction, I.PREC_FP32, w.params, stream=stream)
        g32.set_geometry(w.spheres, w.x3_cap)
        g32.set_state(mid[0], mid[1], 0.0, 0.01)
        set_tiles(g32, args.tiles)
        s32 = timed_window(torch, pf, g32, mid, args.steps, args.warmup, stream, barrier)
        prof32 = g32.profile_stages(3)
        s32_0 = timed_window(torch, pf, g32, t0_state, args.steps, args.warmup, stream, barrier)
        att32 = s32["attempts"]
        top32 = int(np.argmax(prof32[:5]))
        gbs32 = BYTES_F32[top32] * w.n_cells / (prof32[top32] * 1e-3) / 1e9
        forms["fp32_fields"] = {
            "value": w.n_cells * 5 * att32 / (s32["ms"] * 1e-3), "unit": UNIT, "ms_per_step": s32["ms"] / max(att32, 1),
            "window": "midfront",
            "t0_value": w.n_cells * 5 * s32_0["attempts"] / (s32_0["ms"] * 1e-3),
            "gpu_launches": s32["launches"], "dtype": "f32 fields / f64 state", "tiles_by_zc": list(g32.get_tiles()),
            "roofline": {"bound": "hbm", "kernel": f"merson_{stage_names[top32]}_full_sigmap1p_f32",
                         "achieved": gbs32, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                         "frac": gbs32 / peaks["hbm_gbs"],
                         "step_gbs": sum(BYTES_F32) * w.n_cells / (sum(prof32[:5]) * 1e-3) / 1e9,
                         "step_frac": sum(BYTES_F32) * w.n_cells / (sum(prof32[:5]) * 1e-3) / 1e9 / peaks["hbm_gbs"],
                         "traffic": (TRAFFIC_F32_S5_PER_CELL * w.n_cells if (top32 == 4 and TRAFFIC_F32_S5_PER_CELL) else None),
                         "peak_source": peak_kind,
                         "stage_ms": dict(zip(stage_names, prof32))}}
        g32.close()

    study = cycle = None
    if rank == 0 and args.workload == "full512" and not args.no_crop_study:
        study = crop_study(pf, w)
    if rank == 0 and args.workload == "full512" and not args.no_cycle and not args.no_fp32_form:
        cycle = cycle_study(pf, w, stream, {"f64": tiles, "f32_fields": forms["fp32_fields"]["tiles_by_zc"]})

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_sample(w)

    if rank == 0:
        cfg = {"workload": w.name, "grid": list(w.shape), "h_m": w.h, "model": "full",
               "reaction": "SigmaP1-P", "beads": int(w.extra["n_spheres"]),
               "solid_fraction": round(w.extra["solid_fraction_sharp"], 4), "tol": TOL,
               "window": "midfront: freezing front at half height (tanh profile in the pores), "
                         f"{attempts} adaptive attempts after {args.warmup} warm-up attempts",
               "attempts": attempts, "accepted": s["n_accepted"],
               "l2": f"inputs larger than L2 (about {24 * 8 * w.n_cells / 1e9:.0f} GB working set)",
               "tiles_by_zc": list(tiles),
               "parallelism": "replicas" if world > 1 else "single GPU"}
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_max / max(attempts, 1), "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": cfg, "windows": windows,
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
                "clocks": clk.summary(), "forms": forms, "wall_s_timed": t_wall}
        if study:
            line["crop_error_study"] = study
        if cycle:
            line["cycle_time_to_solution"] = cycle
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
