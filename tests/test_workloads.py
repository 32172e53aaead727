"""The input recipes the benchmark and the discharge study state: the
uneven batched sweep and the 32 runs of the Sec. 3.1 study.  These pin the
numbers quoted for them (ranges, time-step rules, capacity), so that a change
to a recipe shows up here and not only in a benchmark line."""
import math

import numpy as np

import workloads

E, ME, EPS0 = 1.602176634e-19, 9.1093837015e-31, 8.8541878128e-12


def _wp(n0):
    return math.sqrt(n0 * E * E / (EPS0 * ME))


def test_batch_sweep_ranges_and_time_steps():
    specs = workloads.batch_configs(256)
    cfgs = workloads.batch_discharges(256)
    assert len(specs) == len(cfgs) == 256
    cells = np.array([s["n_cells"] for s in specs])
    nps = np.array([s["np_init"] for s in specs])
    assert cells.min() >= 64 and cells.max() <= 1024
    assert nps.min() >= 1e4 * 0.999 and nps.max() <= 2e6 * 1.001
    assert len({c["seed"] for c in cfgs}) == 256  # every run its own Philox key
    for s, c in zip(specs, cfgs):
        assert 10.0 <= s["pressure_mtorr"] <= 100.0 and 100.0 <= s["rf_volt"] <= 500.0
        dx = c["length"] / c["n_cells"]
        lam = math.sqrt(EPS0 * c["te_ev"] / (c["n0"] * E))
        assert 0.5 <= dx / lam <= 10.0 + 1e-9
        wpdt = _wp(c["n0"]) * c["dt"]
        assert c["cap_factor"] == 4.0
        if c["scheme"] == "ec_explicit":
            # leapfrog well inside Eq. (1), and a quarter cell per step at v_th
            vth = math.sqrt(E * c["te_ev"] / ME)
            assert wpdt <= 0.2 + 1e-12 and vth * c["dt"] <= 0.25 * dx * (1 + 1e-12)
        else:
            assert c["scheme"] == "ec_implicit"
            assert 0.5 - 1e-9 <= wpdt <= 2.0 + 1e-9
    assert sum(c["scheme"] == "ec_implicit" for c in cfgs) == 128


def test_discharge_study_runs_follow_the_paper_shape():
    from workloads.study import study_runs, F_PAPER, DT_PAPER
    runs = study_runs()
    assert len(runs) == 32
    groups = {}
    for r in runs:
        c = r["cfg"]
        groups.setdefault(r["group"], []).append(r)
        # Sec. 3: 4 cm argon gap, 27 MHz, 200 V, 50 mTorr, 2e16 m^-3 uniform start
        assert c["length"] == 0.04 and c["rf_freq"] == F_PAPER == 27.0e6
        assert c["rf_volt"] == 200.0 and c["pressure_mtorr"] == 50.0 and c["n0"] == 2.0e16
        assert c["np_init"] == r["ppc"] * r["cells"]
        assert c["dt"] == r["dt"]
    assert DT_PAPER == 1.5e-11
    grid = groups["grid"]
    assert sorted((r["scheme"], r["cells"]) for r in grid) == sorted(
        [(s, n) for s in ("ec_explicit", "ec_implicit") for n in (800, 400, 200, 64)]
        + [("mc_explicit", n) for n in (800, 200, 64)] + [("mc_implicit", 400)])
    assert all(r["dt"] == 1.5e-11 and r["ppc"] == 400 for r in grid)
    assert sorted((r["scheme"], r["dt"]) for r in groups["dt"]) == sorted(
        (s, d) for s in ("ec_explicit", "ec_implicit") for d in (1.5e-11, 3e-11, 6e-11, 1e-10))
    assert all(r["cells"] == 100 for r in groups["dt"])
    assert sorted((r["scheme"], r["cells"], r["ppc"]) for r in groups["ppc"]) == sorted(
        (s, n, p) for s in ("ec_explicit", "ec_implicit") for n in (100, 200) for p in (400, 600, 800))
    assert len({r["cfg"]["seed"] for r in runs}) == 32


def test_stretched_benchmark_grid():
    """The stretched form of the production workload: 512 widths summing to
    the 6.7 cm gap, 0.5x the uniform width at the electrodes and 1.5x
    mid-gap (beta = 0.5), symmetric about the middle; everything else as the
    uniform workload."""
    c = workloads.CFG_WIDE_STRETCHED
    u = workloads.CFG_WIDE_EXPLICIT
    h = np.asarray(c["cell_width"])
    dx = u["length"] / u["n_cells"]
    assert h.size == 512 and abs(h.sum() - u["length"]) <= 1e-12 * u["length"]
    assert abs(h[0] / dx - 0.5) < 0.01 and abs(h[255] / dx - 1.5) < 0.01
    assert np.allclose(h, h[::-1], rtol=1e-10)
    for key in ("n_cells", "np_init", "n0", "rf_volt", "rf_freq", "dt", "pressure_mtorr", "sort_period", "scheme"):
        assert c[key] == u[key], key


def test_grid_study_runs():
    """The multi-scale grid study: the paper's discharge with 320 000
    macro-particles per species on 800 and 200 uniform cells and on 200 and
    100 stretched cells (beta = 0.75) whose electrode cells match the 800-
    and 400-cell widths."""
    from workloads.grid_study import grid_runs, NP
    runs = grid_runs()
    assert [(r["cells"], r["beta"]) for r in runs] == [(800, None), (200, None), (200, 0.75), (100, 0.75)]
    for r in runs:
        c = r["cfg"]
        assert c["np_init"] == NP == 320_000 and c["scheme"] == "ec_explicit"
        assert c["length"] == 0.04 and c["rf_freq"] == 27.0e6 and c["dt"] == 1.5e-11
        if r["beta"] is not None:
            h = np.asarray(c["cell_width"])
            assert abs(h.sum() - 0.04) < 1e-15 and abs(h[0] / (0.04 / (4 * c["n_cells"])) - 1.0) < 0.01
    assert len({r["cfg"]["seed"] for r in runs}) == 4
