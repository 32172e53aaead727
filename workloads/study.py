"""The discharge study of Sec. 3.1 rerun with the library, qualitatively.

    python -m workloads.study [--periods 1800] [--avg-periods 300] [--out workloads/discharge_study.json]

The paper's benchmark discharge (Sec. 3: 4 cm argon gap, 27 MHz, 200 V on one
electrode, 50 mTorr, 2e16 m^-3 uniform start, 400 macro-particles per cell,
dt = 1.5e-11 s) run as one batch of independent runs through pic_batch_*:
  * grid spacing (the figures of densities, potential, sheath, heating and
    EEPF): EC explicit and EC direct implicit with 800, 400, 200 and 64 cells;
    the momentum-conserving explicit scheme with 800 cells (the paper's
    benchmark), 200 and 64 cells (where it is expected to self-heat), and the
    momentum-conserving implicit scheme with 400 cells;
  * time step at 100 cells: dt = 1.5e-11, 3e-11, 6e-11 and 1e-10 s, EC explicit
    and EC implicit;
  * macro-particles per cell at 100 and 200 cells: 400, 600 and 800, EC
    explicit and EC implicit.
Every run starts from its own uniform Maxwellian load and advances
`periods` RF periods of its own dt; the time averages (densities, potential,
J.E heating, EEDF) are taken over the last `avg_periods`.  The analytic
stand-in cross sections replace the paper's argon set, and the runs are far
shorter than the paper's converged ones, so the study compares shapes and
trends, not values.  Profiles are stored on at most 100 points.
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


def study_runs() -> list[dict]:
    runs = []

    def add(group, scheme, cells, dt=DT_PAPER, ppc=400):
        c = workloads.cfg_paper(cells, scheme)
        c.update(np_init=ppc * cells, dt=dt, diag_period=20, eedf_bins=60, eedf_max_ev=30.0,
                 sort_period=16, cap_factor=3.0, seed=100 + len(runs), run=len(runs),
                 name="%s_%s_%dcells_dt%.3g_ppc%d" % (group, scheme, cells, dt, ppc))
        runs.append(dict(group=group, scheme=scheme, cells=cells, dt=dt, ppc=ppc, cfg=c))

    for scheme in ("ec_explicit", "ec_implicit"):
        for cells in (800, 400, 200, 64):
            add("grid", scheme, cells)
    for cells in (800, 200, 64):
        add("grid", "mc_explicit", cells)
    add("grid", "mc_implicit", 400)
    for scheme in ("ec_explicit", "ec_implicit"):
        for dt in (1.5e-11, 3e-11, 6e-11, 1e-10):
            add("dt", scheme, 100, dt=dt)
    for scheme in ("ec_explicit", "ec_implicit"):
        for cells in (100, 200):
            for ppc in (400, 600, 800):
                add("ppc", scheme, cells, ppc=ppc)
    return runs


def _coarse(a, n=100):
    a = np.asarray(a, dtype=np.float64)
    if len(a) <= n:
        return a.tolist()
    edges = np.linspace(0, len(a), n + 1).astype(int)
    return [float(a[i:j].mean()) for i, j in zip(edges[:-1], edges[1:])]


def _summary(r, prof, cfg):
    """Scalar features of one run's averaged profiles."""
    L = cfg["length"]
    n = cfg["n_cells"]
    dx = L / n
    ne, ni = prof["ne"], prof["ni"]
    mid = slice(int(0.4 * n), int(0.6 * n) + 1)
    dn = ni - ne
    # sheath edge at each electrode: first node from the wall where n_e
    # reaches half of n_i (the quasi-neutral edge)
    def edge(order):
        for g in order:
            if ni[g] > 0 and ne[g] >= 0.5 * ni[g]:
                return g
        return None
    e0 = edge(range(0, n + 1))
    e1 = edge(range(n, -1, -1))
    eedf = prof["eedf"].astype(np.float64)
    bins = len(eedf) - 1
    width = cfg["eedf_max_ev"] / bins
    centres = (np.arange(bins) + 0.5) * width
    tot = max(eedf.sum(), 1.0)
    he = prof["heat_e"]
    return {
        "ne_mid": float(ne[mid].mean()), "ni_mid": float(ni[mid].mean()),
        "phi_mid": float(prof["phi"][mid].mean()),
        "sheath_left_m": None if e0 is None else e0 * dx, "sheath_right_m": None if e1 is None else (n - e1) * dx,
        "dn_max": float(dn.max()),
        "heat_e_peak": float(he.max()), "heat_e_total_w_m2": float(he.sum() * dx),
        "heat_e_bulk_w_m3": float(he[mid].mean()),
        "heat_i_total_w_m2": float(prof["heat_i"].sum() * dx),
        "eedf_mean_ev": float((eedf[:bins] * centres).sum() / max(eedf[:bins].sum(), 1.0)),
        "eedf_frac_above_15ev": float(eedf[int(15.0 / width):].sum() / tot),
    }


def run_study(periods: int, avg_periods: int, device="cuda:0") -> dict:
    import torch
    from paper_1310_5284_gb300.batch import BatchSim

    runs = study_runs()
    cfgs = [r["cfg"] for r in runs]
    batch = BatchSim(cfgs, device=device)
    steps_total = int(round(periods / (F_PAPER * DT_PAPER)))
    steps_avg = int(round(avg_periods / (F_PAPER * DT_PAPER)))
    chunk = 20 * int(round(1.0 / (F_PAPER * DT_PAPER)))  # 20 periods per call
    history = {i: [] for i in range(len(runs))}
    t0 = time.time()
    done = 0
    while done < steps_total - steps_avg:
        n = min(chunk, steps_total - steps_avg - done)
        batch.step(n)
        done += n
        for i in range(len(runs)):
            history[i].append(sum(batch.diag(i)["count"]) // 2)
    for i in range(len(runs)):
        batch.diag(i, reset_avg=True)
    while done < steps_total:
        n = min(chunk, steps_total - done)
        batch.step(n)
        done += n
        for i in range(len(runs)):
            history[i].append(sum(batch.diag(i)["count"]) // 2)
    torch.cuda.synchronize()
    wall = time.time() - t0
    out = {"periods": periods, "avg_periods": avg_periods, "steps": steps_total, "wall_s": wall,
           "status": batch.status(), "runs": []}
    for i, r in enumerate(runs):
        prof = batch.profiles(i)
        d = batch.diag(i)
        cfg = r["cfg"]
        out["runs"].append({
            "group": r["group"], "scheme": r["scheme"], "cells": r["cells"], "dt": r["dt"], "ppc": r["ppc"],
            "dx_over_debye_at_load": cfg["length"] / cfg["n_cells"] /
            math.sqrt(8.8541878128e-12 * cfg["te_ev"] / (cfg["n0"] * 1.602176634e-19)),
            "status": d["status"], "count": d["count"], "electrons_every_20_periods": history[i],
            "summary": _summary(r, prof, cfg),
            "x_m": _coarse(np.linspace(0.0, cfg["length"], cfg["n_cells"] + 1)),
            "ne": _coarse(prof["ne"]), "ni": _coarse(prof["ni"]), "phi": _coarse(prof["phi"]),
            "heat_e": _coarse(prof["heat_e"]), "heat_i": _coarse(prof["heat_i"]),
            "eedf": prof["eedf"].astype(np.int64).tolist(),
        })
    batch.close()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--periods", type=int, default=1800)
    ap.add_argument("--avg-periods", type=int, default=300)
    ap.add_argument("--out", default=os.path.join(os.path.dirname(os.path.abspath(__file__)),
                                                  "discharge_study.json"))
    a = ap.parse_args()
    res = run_study(a.periods, a.avg_periods)
    with open(a.out, "w") as f:
        json.dump(res, f)
    print(json.dumps({"wall_s": res["wall_s"], "status": res["status"],
                      "runs": [(r["group"], r["scheme"], r["cells"], r["dt"], r["ppc"], r["status"],
                                round(r["summary"]["ne_mid"] / 1e16, 3)) for r in res["runs"]]}))


if __name__ == "__main__":
    main()
