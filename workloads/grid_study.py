"""The multi-scale grid Sec. 4 proposes, tried on the paper's benchmark
discharge (qualitatively).

    python -m workloads.grid_study [--periods 600] [--avg-periods 200] [--out workloads/grid_study.json]

The paper's discharge (Sec. 3: 4 cm argon gap, 27 MHz, 200 V, 50 mTorr,
2e16 m^-3 uniform start, dt = 1.5e-11 s, explicit EC scheme) with the same
320 000 macro-particles per species on four grids:
  * 800 uniform cells (the paper's reference grid);
  * 200 uniform cells;
  * 200 stretched cells, beta = 0.75: cells of the 800-cell width at the
    electrodes, 1.75x the 200-cell width mid-gap;
  * 100 stretched cells, beta = 0.75: the 400-cell width at the electrodes.
Each run starts from its own uniform load and advances `periods` RF periods;
the time averages are taken over the last `avg_periods`.  The analytic
stand-in cross sections replace the paper's argon set and the runs are far
shorter than converged ones, so the study compares the grids with one
another, not with the paper's values.  Profiles are stored on at most 100
points of the node positions.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import time

import numpy as np

import workloads

F_PAPER = 27.0e6
DT_PAPER = 1.5e-11
NP = 320_000  # macro-particles per species in every run (400 per cell at 800 cells)


def grid_runs() -> list[dict]:
    runs = []
    for cells, beta in ((800, None), (200, None), (200, 0.75), (100, 0.75)):
        c = workloads.cfg_paper(cells, "ec_explicit")
        c.update(np_init=NP, diag_period=20, eedf_bins=60, eedf_max_ev=30.0, sort_period=16, cap_factor=3.0,
                 seed=500 + len(runs))
        if beta is not None:
            c = workloads.with_stretch(c, beta)
        c["name"] = "paper_%dcells_%s" % (cells, "uniform" if beta is None else "stretched%g" % beta)
        runs.append(dict(cells=cells, beta=beta, cfg=c))
    return runs


def _nodes(cfg) -> np.ndarray:
    if cfg.get("cell_width") is None:
        return np.linspace(0.0, cfg["length"], cfg["n_cells"] + 1)
    return np.concatenate([[0.0], np.cumsum(cfg["cell_width"])])


def _coarse(x, a, n=100):
    """The profile a(x) on n + 1 evenly spaced points of the gap."""
    xs = np.linspace(x[0], x[-1], n + 1)
    return np.interp(xs, x, np.asarray(a, dtype=np.float64)).tolist()


def _summary(prof, cfg):
    x = _nodes(cfg)
    n = cfg["n_cells"]
    length = cfg["length"]
    ne, ni = prof["ne"], prof["ni"]
    mid = (x >= 0.4 * length) & (x <= 0.6 * length)

    # sheath edge at each electrode: first node from the wall where n_e
    # reaches half of n_i (the quasi-neutral edge)
    def edge(order):
        for g in order:
            if ni[g] > 0 and ne[g] >= 0.5 * ni[g]:
                return g
        return None

    e0 = edge(range(0, n + 1))
    e1 = edge(range(n, -1, -1))
    h = np.diff(x)
    he = prof["heat_e"]
    eedf = prof["eedf"].astype(np.float64)
    bins = len(eedf) - 1
    width = cfg["eedf_max_ev"] / bins
    centres = (np.arange(bins) + 0.5) * width
    return {
        "ne_mid": float(ne[mid].mean()), "ni_mid": float(ni[mid].mean()),
        "phi_mid": float(prof["phi"][mid].mean()),
        "sheath_left_m": None if e0 is None else float(x[e0]),
        "sheath_right_m": None if e1 is None else float(length - x[e1]),
        "electrode_cell_m": float(h[0]), "mid_cell_m": float(h[n // 2]),
        "heat_e_total_w_m2": float((he * h).sum()), "heat_i_total_w_m2": float((prof["heat_i"] * h).sum()),
        "eedf_mean_ev": float((eedf[:bins] * centres).sum() / max(eedf[:bins].sum(), 1.0)),
    }


def run_grid_study(periods: int, avg_periods: int, device="cuda:0") -> dict:
    import torch
    from paper_1310_5284_gb300.sim import Sim

    steps_per_period = int(round(1.0 / (F_PAPER * DT_PAPER)))
    out = {"periods": periods, "avg_periods": avg_periods, "steps": periods * steps_per_period, "runs": []}
    for r in grid_runs():
        cfg = r["cfg"]
        sim = Sim(cfg, device=device)
        t0 = time.time()
        sim.step((periods - avg_periods) * steps_per_period)
        sim.diag(reset_avg=True)
        sim.step(avg_periods * steps_per_period)
        d = sim.diag()
        torch.cuda.synchronize()
        wall = time.time() - t0
        prof = sim.profiles()
        x = _nodes(cfg)
        lam = math.sqrt(8.8541878128e-12 * cfg["te_ev"] / (cfg["n0"] * 1.602176634e-19))
        out["runs"].append({
            "name": cfg["name"], "cells": r["cells"], "beta": r["beta"], "status": d["status"],
            "count": d["count"], "wall_s": wall,
            "cell_over_debye_at_load": [float(np.diff(x).min() / lam), float(np.diff(x).max() / lam)],
            "summary": _summary(prof, cfg),
            "ne": _coarse(x, prof["ne"]), "ni": _coarse(x, prof["ni"]), "phi": _coarse(x, prof["phi"]),
            "eedf": prof["eedf"].astype(np.int64).tolist(),
        })
        sim.close()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--periods", type=int, default=600)
    ap.add_argument("--avg-periods", type=int, default=200)
    ap.add_argument("--out", default=os.path.join(os.path.dirname(os.path.abspath(__file__)), "grid_study.json"))
    a = ap.parse_args()
    res = run_grid_study(a.periods, a.avg_periods)
    with open(a.out, "w") as f:
        json.dump(res, f)
    print(json.dumps([(r["name"], r["status"], round(r["wall_s"], 1), {k: (None if v is None else float("%.4g" % v))
                                                                        for k, v in r["summary"].items()})
                      for r in res["runs"]]))


if __name__ == "__main__":
    main()
