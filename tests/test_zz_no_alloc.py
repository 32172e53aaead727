"""pic_deposit_noalloc: charge assignment for callers that cannot allocate
device memory where they need a density (inside another framework's memory
pool, in allocation-free real-time loops, in tools that hold only particle
arrays).  Its per-node sums live in the library's static device array, so
the call needs nothing but its inputs and output.  Checked against the run
path (pic_set_particles + pic_init_field + pic_grids) on two calls in a row:
the second call must not see the first call's sums.  This file is named to
be collected last."""
import ctypes

import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu


def _vth(cfg, k):
    e, me, amu = 1.602176634e-19, 9.1093837015e-31, 1.66053906660e-27
    return (e * (cfg["te_ev"] if k == 0 else cfg["ti_ev"]) / (me if k == 0 else cfg["ion_mass_amu"] * amu)) ** 0.5


def test_noalloc_deposit_matches_run_path_on_consecutive_calls():
    import torch

    import __graft_entry__
    __graft_entry__.build()
    from paper_1310_5284_gb300 import _abi
    from paper_1310_5284_gb300.sim import Sim

    lib = _abi.lib()
    stream = torch.cuda.current_stream()
    cases = [
        ("ec_electrodes_97", dict(n_cells=97), 40_001, 0, 0),
        ("ec_periodic_64", dict(n_cells=64, periodic=True, rf_volt=0.0), 12_345, 0, 1),
        ("mc_electrodes_33", dict(n_cells=33, scheme="mc_explicit"), 7_777, 1, 0),
        ("mc_periodic_29", dict(n_cells=29, periodic=True, rf_volt=0.0, scheme="mc_explicit"), 5_003, 1, 1),
        ("ec_implicit_electrodes_50", dict(n_cells=50, scheme="ec_implicit", dt=8e-10), 9_001, 2, 0),
        ("mc_implicit_periodic_41", dict(n_cells=41, periodic=True, rf_volt=0.0, scheme="mc_implicit",
                                         dt=8e-10), 6_007, 3, 1),
    ]
    for name, over, n, scheme, boundary in cases:
        cfg = dict(workloads.CFG_SMALL_CCP, mcc=False, np_init=n)
        cfg.update(over)
        st_e = workloads.injected_particles(300 + n, n, cfg["n_cells"], _vth(cfg, 0))
        st_i = workloads.injected_particles(301 + n, n, cfg["n_cells"], _vth(cfg, 1))
        sim = Sim(cfg)
        sim.set_particles("e", st_e)
        sim.set_particles("i", st_i)
        sim.init_field()
        ref = sim.grids()
        sim.close()
        for species, st in (("rho_q_e", st_e), ("rho_q_i", st_i)):
            cell = torch.from_numpy(st["cell"]).cuda()
            off = torch.from_numpy(st["off"]).cuda()
            out = torch.full((cfg["n_cells"] + 1,), -1, dtype=torch.int64, device="cuda")
            rc = lib.pic_deposit_noalloc(scheme, boundary, cfg["n_cells"], cell.data_ptr(), off.data_ptr(), n,
                                         out.data_ptr(), ctypes.c_void_p(stream.cuda_stream))
            torch.cuda.synchronize()
            assert rc == 0, lib.pic_last_error(None)
            got = out.cpu().numpy()
            assert np.array_equal(got, ref[species]), (name, species)
            assert got.sum() == n * 2 ** 33


def test_noalloc_deposit_rejects_grids_beyond_the_static_scratch():
    import torch

    from paper_1310_5284_gb300 import _abi

    lib = _abi.lib()
    out = torch.zeros(2050, dtype=torch.int64, device="cuda")
    cell = torch.zeros(4, dtype=torch.int32, device="cuda")
    off = torch.zeros(4, dtype=torch.float32, device="cuda")
    rc = lib.pic_deposit_noalloc(0, 0, 2048, cell.data_ptr(), off.data_ptr(), 4, out.data_ptr(), None)
    assert rc == -1
    assert b"1024" in lib.pic_last_error(None)


def _call(lib, scheme, boundary, n_cells, cell, off, n, out, stream):
    return lib.pic_deposit_noalloc(scheme, boundary, n_cells, cell, off, n, out,
                                   ctypes.c_void_p(stream.cuda_stream))


def test_noalloc_deposit_skips_entries_off_the_grid_and_clears_between_calls():
    """Entries with a cell outside the grid or an offset outside [0, 1)
    (-0.1, 1.0, NaN) assign nothing: the result equals the run path's for the
    other particles.  A call with no particles returns all zeros, also right
    after a call that filled the static sums."""
    import torch

    import __graft_entry__
    __graft_entry__.build()
    from paper_1310_5284_gb300 import _abi
    from paper_1310_5284_gb300.sim import Sim

    lib = _abi.lib()
    stream = torch.cuda.current_stream()
    cfg = dict(workloads.CFG_SMALL_CCP, mcc=False, np_init=3000, n_cells=40)
    n = cfg["np_init"]
    st = workloads.injected_particles(4242, n, cfg["n_cells"], _vth(cfg, 0))
    bad = np.array([5, 77, 1234, 2000, 2999])
    cell = st["cell"].copy()
    off = st["off"].copy()
    off[bad[0]] = np.float32(-0.1)
    off[bad[1]] = np.float32(1.0)
    off[bad[2]] = np.float32(np.nan)
    cell[bad[3]] = -1
    cell[bad[4]] = cfg["n_cells"]
    keep = np.setdiff1d(np.arange(n), bad)
    for scheme, sch_name in ((0, "ec_explicit"), (1, "mc_explicit")):
        sim = Sim(dict(cfg, scheme=sch_name, np_init=len(keep)))
        sim.set_particles("e", {k: v[keep] for k, v in st.items()})
        sim.init_field()
        ref = sim.grids()["rho_q_e"]
        sim.close()
        c_d = torch.from_numpy(cell).cuda()
        o_d = torch.from_numpy(off).cuda()
        out = torch.full((cfg["n_cells"] + 1,), -1, dtype=torch.int64, device="cuda")
        rc = _call(lib, scheme, 0, cfg["n_cells"], c_d.data_ptr(), o_d.data_ptr(), n, out.data_ptr(), stream)
        torch.cuda.synchronize()
        assert rc == 0, lib.pic_last_error(None)
        got = out.cpu().numpy()
        assert np.array_equal(got, ref), sch_name
        assert got.sum() == len(keep) * 2 ** 33
        # no particles: all zeros, twice (the sums of the call above are gone)
        for _ in range(2):
            out.fill_(-7)
            rc = _call(lib, scheme, 0, cfg["n_cells"], None, None, 0, out.data_ptr(), stream)
            torch.cuda.synchronize()
            assert rc == 0, lib.pic_last_error(None)
            assert not out.cpu().numpy().any()
