"""Batched persistent runs against the same configurations run alone: every
particle bit-identical (charge sums are integers and draws are keyed on
(id, step, run), so neither the work split nor the schedule can change a
result), whatever the work-item size and sort period."""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def batch_cases():
    base = dict(workloads.CFG_SMALL_CCP)
    return [
        dict(base, n_cells=64, np_init=3000, seed=11, run=0),
        dict(base, n_cells=97, np_init=5001, scheme="mc_explicit", seed=12, run=1),
        dict(base, n_cells=50, np_init=4000, scheme="ec_implicit", dt=8e-10, seed=13, run=2),
        dict(workloads.cfg_periodic(n_cells=40, np_e=2000, n0=1e15, length=0.02, dt=5e-11), seed=14, run=3),
        dict(base, n_cells=200, np_init=20000, te_ev=6.0, seed=15, run=4),
        dict(base, n_cells=33, np_init=700, scheme="ec_implicit", dt=6e-10, te_ev=5.0, seed=16, run=5),
        dict(base, n_cells=1024, np_init=9000, seed=17, run=6, sort_period=4),
        dict(base, n_cells=71, np_init=6000, scheme="mc_implicit", dt=5e-10, te_ev=6.0, seed=18, run=7),
    ]


def by_id(d):
    o = np.argsort(d["id"])
    return {k: v[o] for k, v in d.items() if isinstance(v, np.ndarray)}


def test_batched_runs_bit_identical_to_single_runs():
    from paper_1310_5284_gb300.batch import BatchSim
    from paper_1310_5284_gb300.sim import Sim

    cfgs = batch_cases()
    batch = BatchSim(cfgs)
    batch.step(17)
    batch.set_schedule(1024, 4)  # a different work split and sort period mid-run
    batch.step(23)
    assert batch.status() == 0
    for r, cfg in enumerate(cfgs):
        single = Sim(cfg)
        single.step(40)
        db, ds = batch.diag(r), single.diag()
        assert db["step"] == ds["step"] == 40
        assert db["count"] == ds["count"], r
        assert db["coll"] == ds["coll"] and db["births"] == ds["births"], r
        for sp in ("e", "i"):
            a, b = by_id(batch.get_particles(r, sp)), by_id(single.get_particles(sp))
            for key in ("id", "cell", "off", "vx", "vy", "vz"):
                assert np.array_equal(a[key], b[key]), (r, sp, key)
            if cfg.get("scheme") in ("ec_implicit", "mc_implicit"):
                assert np.array_equal(a["abar"], b["abar"]), (r, sp)
        single.close()
    batch.close()


def test_batch_autotune_keeps_results():
    from paper_1310_5284_gb300.batch import BatchSim
    from paper_1310_5284_gb300.sim import Sim

    cfgs = batch_cases()[:4]
    batch = BatchSim(cfgs)
    best = batch.autotune(trial_steps=4)
    assert best["chunk"] >= 4096 and best["sort_period"] in (4, 8, 16, 32) and best["ms_per_step"] > 0
    steps = batch.diag(0)["step"]
    batch.step(8)
    for r, cfg in enumerate(cfgs):
        single = Sim(cfg)
        single.step(steps + 8)
        for sp in ("e", "i"):
            a, b = by_id(batch.get_particles(r, sp)), by_id(single.get_particles(sp))
            for key in ("id", "cell", "off", "vx", "vy", "vz"):
                assert np.array_equal(a[key], b[key]), (r, sp, key)
        single.close()


def test_batch_profiles_equal_the_single_run_profiles():
    """pic_batch_profiles: the time-averaged densities, potential, heating
    profiles and EEDF of each batched run, after a reset and 30 steps with
    diagnostics every 3 steps, equal those of the same run alone (the runs are
    bit-identical; the FP64 averages are summed in the same order)."""
    from paper_1310_5284_gb300.batch import BatchSim
    from paper_1310_5284_gb300.sim import Sim

    cfgs = [dict(c, diag_period=3, eedf_bins=32) for c in batch_cases()[:5]]
    batch = BatchSim(cfgs)
    batch.step(9)
    for r in range(len(cfgs)):
        batch.diag(r, reset_avg=True)
    batch.step(30)
    for r, cfg in enumerate(cfgs):
        single = Sim(cfg)
        single.step(9)
        single.diag(reset_avg=True)
        single.step(30)
        pb, ps = batch.profiles(r), single.profiles()
        for key in ("ne", "ni", "phi", "eedf"):
            assert np.array_equal(pb[key], ps[key]), (r, key)
        for key in ("heat_e", "heat_i"):  # per-block FP32 heating sums: order of blocks may differ
            np.testing.assert_allclose(pb[key], ps[key], rtol=1e-5, atol=1e-6 * max(np.abs(ps[key]).max(), 1e-30))
        assert pb["ne"].sum() > 0
        single.close()
    batch.close()


def test_benchmark_sweep_stays_clean_over_its_window():
    """The 256 uneven runs the benchmark times (cells 64..1024, 1e4..2e6
    particles per species, explicit and direct implicit) over the benchmark's
    2000 steps: no run drops a birth or a particle (its status word stays 0)
    and none grows beyond three times its load, so the throughput is that of
    discharges in regime."""
    from paper_1310_5284_gb300.batch import BatchSim

    cfgs = workloads.batch_discharges(256)
    batch = BatchSim(cfgs)
    c0 = [sum(batch.diag(i)["count"]) for i in range(len(cfgs))]
    batch.step(2000)
    assert batch.status() == 0
    for i in range(len(cfgs)):
        d = batch.diag(i)
        assert d["status"] == 0, (i, d["status"])
        assert d["step"] == 2000
        assert sum(d["count"]) <= 3 * c0[i], (i, sum(d["count"]), c0[i])
    batch.close()
