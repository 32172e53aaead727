"""Discharge statistics of the GPU run against the same run in the FP64 oracle.

The two runs start from the same load and draw from the same Philox streams,
but the plasma's chaos separates their trajectories within tens of steps, so
only statistics can agree.  Case: the small CCP (2 cm, 64 cells, 200 V,
13.56 MHz, 30 mTorr) with 51,200 macro-particles per species, 10 RF cycles
after the load, then averages over 50 cycles.

Bars.  Ion wall fluxes at both electrodes, the time-averaged electron and ion
density profiles (relative L2 norm over the nodes) and the EEDF (L1 distance
of the normalised histograms) and mean electron energy: 2 %.  The rest are set
about 1.5x above the largest spread between oracle runs that differ only in
their seed (four seeds, six pairs, this window): time-averaged potential
(seed spread <= 0.13 %, bar 2 %), ion J.E heating profile (<= 1.5 %, bar 3 %),
power absorbed by the ions (<= 0.7 %, bar 2 %), ion wall energy (<= 2.2 %, bar
4 %); the electron quantities of a discharge ten cycles after a uniform load
are far from converged and spread more: electron wall counts (<= 6.9 %, bar
10 %), electron wall energy (<= 7.1 %, bar 11 %), electron J.E heating profile
summed over 8-cell bins (<= 5.5 %, bar 9 %) and power absorbed by the
electrons (<= 6.3 %, bar 10 %).  The GPU and oracle runs share their load and
Philox streams, so they differ less than two seeds do.  Each diagnostic's
arithmetic is checked step by step, without chaos, at 1e-5 or better in
test_gpu_parity.py (one_step_diagnostics).
"""
import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu

STEPS_PER_CYCLE = 400
WARM_CYCLES, WINDOW_CYCLES = 10, 50
EEDF_BINS, EEDF_MAX = 60, 30.0


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def case():
    return dict(workloads.CFG_SMALL_CCP, np_init=51200, diag_period=10, eedf_bins=EEDF_BINS,
                eedf_max_ev=EEDF_MAX, sort_period=16)


def run(sim):
    sim.step(STEPS_PER_CYCLE * WARM_CYCLES)
    sim.reset_averages() if hasattr(sim, "reset_averages") else sim.diag(reset_avg=True)
    d0 = sim.diag()
    sim.step(STEPS_PER_CYCLE * WINDOW_CYCLES)
    d1 = sim.diag()
    av = sim.averages() if hasattr(sim, "averages") else sim.profiles()
    wall = np.array(d1["wall_count"], dtype=np.float64) - np.array(d0["wall_count"], dtype=np.float64)
    energy = np.array(d1["wall_energy_ev"], dtype=np.float64) - np.array(d0["wall_energy_ev"], dtype=np.float64)
    return wall, energy, av


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def bins(h, width=8):
    n = len(h) // width * width
    return np.asarray(h[:n]).reshape(-1, width).sum(axis=1)


def test_window_statistics_match_oracle():
    from paper_1310_5284_gb300.sim import Sim

    cfg = case()
    n = cfg["np_init"]
    gpu = Sim(cfg, device="cuda:0")
    w_g, en_g, a_g = run(gpu)
    assert gpu.status() == 0
    gpu.close()
    orc = oracle.Sim(dict(cfg, quantized=True)).load(n, n)
    w_o, en_o, a_o = run(orc)
    dx = cfg["length"] / cfg["n_cells"]

    rel_wall = np.abs(w_g - w_o) / w_o
    print("wall counts gpu", w_g.tolist(), "oracle", w_o.tolist(), "rel", rel_wall.round(4).tolist())
    assert np.all(w_o > 5000)  # enough events for a 2 % comparison
    assert np.all(rel_wall[1] <= 0.02)  # ions, both electrodes
    assert np.all(rel_wall[0] <= 0.10)  # electrons
    rel_en = np.abs(en_g - en_o) / en_o
    print("wall energy rel", rel_en.round(4).tolist())
    assert np.all(rel_en[1] <= 0.04)
    assert np.all(rel_en[0] <= 0.11)

    for key in ("ne", "ni"):
        err = rel_l2(a_g[key], a_o[key])
        print(key, "profile L2", err)
        assert err <= 0.02, key
    err_phi = rel_l2(a_g["phi"], a_o["phi"])
    print("phi profile L2", err_phi)
    assert err_phi <= 0.02

    err_hi = rel_l2(a_g["heat_i"], a_o["heat_i"])
    err_he = rel_l2(bins(a_g["heat_e"]), bins(a_o["heat_e"]))
    p_g = [float(a_g["heat_e"].sum() * dx), float(a_g["heat_i"].sum() * dx)]
    p_o = [float(a_o["heat_e"].sum() * dx), float(a_o["heat_i"].sum() * dx)]
    print("heating L2 e (8-cell bins)", err_he, "i", err_hi, "power gpu", p_g, "oracle", p_o)
    assert err_hi <= 0.03
    assert err_he <= 0.09
    assert p_o[0] > 0 and p_o[1] > 0  # both species absorb power on average
    assert abs(p_g[1] - p_o[1]) <= 0.02 * p_o[1]
    assert abs(p_g[0] - p_o[0]) <= 0.10 * p_o[0]

    eg = a_g["eedf"].astype(np.float64)
    eo = a_o["eedf"].astype(np.float64)
    eg, eo = eg[:EEDF_BINS] / eg.sum(), eo[:EEDF_BINS] / eo.sum()
    l1 = np.abs(eg - eo).sum()
    centres = (np.arange(EEDF_BINS) + 0.5) * EEDF_MAX / EEDF_BINS
    mean_g, mean_o = (eg * centres).sum() / eg.sum(), (eo * centres).sum() / eo.sum()
    print("eedf L1", l1, "mean energy", mean_g, mean_o)
    assert l1 <= 0.02
    assert abs(mean_g - mean_o) <= 0.02 * mean_o
