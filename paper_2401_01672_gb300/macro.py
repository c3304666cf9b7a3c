"""Macro-scale freeze-thaw runs of the vessel of Sec. 3.1 (Table 2) through the library.

One run integrates one model on the vessel for 5 h of cooling through the cap and 5 h of heating,
stopping at `n_samples` evenly spaced times to record the ice volume fraction |Omega_I| / |Omega_W|
(eqs. water-occupied-subdomain, frozen-subdomain: the library's unfrozen-water counts) and the extreme
phase-field values.  Every step runs in the library's kernels; the host only reads the counts and the
state at the sample times.  A run that fails (non-finite state, step-size underflow) or hits its attempt
cap is reported as such: the paper finds the GradP model unstable at small surface tension.
"""
from __future__ import annotations

import math
import time

import numpy as np

from . import inputs as I
from . import pf


def run_case(w, n_samples=60, tol=1e-6, max_attempts=3_000_000, precision=I.PREC_FP64, dt0=1e-3):
    """Integrate workload `w` (inputs.macro_case) to its end time; returns the ice-fraction curve and
    the run's counters and wall time."""
    import torch
    g = pf.Grid(w.shape, w.h, w.model, w.reaction, precision, w.params)
    try:
        g.set_geometry(w.spheres, w.x3_cap)
        g.set_state(w.theta0 if w.model != I.MODEL_MICRO else None, w.phi0, 0.0, dt0)
        tiles = g.autotune(None)[:2]
        t_end = w.extra["t_end"]
        times = [t_end * (q + 1) / n_samples for q in range(n_samples)]
        curve = []
        attempts = accepted = 0
        status = "ok"
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for ts in times:
            left = max_attempts - attempts
            if left <= 0:
                status = "attempt cap"
                break
            try:
                s = g.run_to(ts, tol, left)
            except pf.PfError as e:
                status = {pf.PF_E_NONFINITE: "non-finite state", pf.PF_E_DT_UNDERFLOW: "step-size underflow"}.get(
                    e.status, f"status {e.status}")
                break
            attempts += s["n_accepted"] + s["n_rejected"]
            accepted += s["n_accepted"]
            u = g.unfrozen_fraction()
            th, ph, t_now, dt = g.get_state()
            curve.append({"t": t_now, "ice_fraction": u["n_ice"] / u["n_water"] if u["n_water"] else math.nan,
                          "phi_min": float(np.min(ph)) if ph is not None else None,
                          "phi_max": float(np.max(ph)) if ph is not None else None,
                          "theta_min": float(np.min(th)), "theta_max": float(np.max(th)), "dt": dt})
            if t_now < ts * (1 - 1e-12):
                status = "attempt cap"
                break
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
    finally:
        g.close()
    return {"name": w.name, "status": status, "wall_s": wall, "attempts": attempts, "accepted": accepted,
            "cells": w.n_cells, "tiles_by_zc": list(tiles), "curve": curve}


def summary(run, t_freeze=I.MACRO_T_FREEZE):
    """Times at which the ice fraction first reaches 1/2 while cooling and falls below 1/2 again while
    heating (None if it does not), and the ice fraction at the end of cooling."""
    c = run["curve"]
    t_half_freeze = next((p["t"] for p in c if p["t"] <= t_freeze + 1e-9 and p["ice_fraction"] >= 0.5), None)
    t_half_thaw = next((p["t"] for p in c if p["t"] > t_freeze + 1e-9 and p["ice_fraction"] < 0.5), None)
    at_freeze = [p["ice_fraction"] for p in c if abs(p["t"] - t_freeze) <= 1e-6 * t_freeze]
    return {"t_half_freeze_s": t_half_freeze, "t_half_thaw_s": t_half_thaw,
            "ice_fraction_end_of_cooling": at_freeze[0] if at_freeze else None,
            "phi_max": max((p["phi_max"] for p in c if p["phi_max"] is not None), default=None)}


def curve_distance(a, b):
    """Largest difference of two runs' ice fractions over their common sample times."""
    tb = {round(p["t"], 6): p["ice_fraction"] for p in b["curve"]}
    d = [abs(p["ice_fraction"] - tb[round(p["t"], 6)]) for p in a["curve"] if round(p["t"], 6) in tb]
    return max(d) if d else None
