"""The explicit EC scheme on a non-uniform grid (the multi-scale grid of
Sec. 4) on the GPU: properties that hold at any size, beside the element-wise
parity cases of test_gpu_parity.py (load, deposit and field, steps,
collisions, sort and graph replay) and test_gpu_fullsize.py.

Energy: a collisionless periodic plasma on cells 5 to 15 Debye lengths wide
keeps its total energy within 1 % over 1000 / omega_p at omega_p dt = 0.1, as
the FP64 oracle does on the same grid (its pin), and the GPU's history stays
within 2x the oracle's own deviation plus 1e-3.
"""
import math

import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu

E = 1.602176634e-19
ME = 9.1093837015e-31
EPS0 = 8.8541878128e-12


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def thermal_cfg(wdt=0.1, beta=0.5):
    n0, te = 1e15, 2.0
    lam = math.sqrt(EPS0 * te / (n0 * E))
    n_cells, ppc = 64, 64
    wp = math.sqrt(n0 * E * E / (EPS0 * ME))
    c = workloads.cfg_periodic_stretched(n_cells=n_cells, np_sp=n_cells * ppc, n0=n0,
                                         length=n_cells * 10 * lam, dt=wdt / wp, te_ev=te, beta=beta)
    return dict(c, sort_period=16)


def test_stretched_grid_conserves_energy_like_the_oracle():
    from paper_1310_5284_gb300.sim import Sim
    cfg = thermal_cfg()
    n = cfg["np_init"]
    gpu = Sim(cfg, device="cuda:0")
    orc = oracle.Sim(dict(cfg, quantized=True)).load(n, n)
    gpu.step(1)
    orc.step(1)
    eg, eo = [gpu.energy()], [orc.energy()]
    for _ in range(100):
        gpu.step(100)
        orc.step(100)
        eg.append(gpu.energy())
        eo.append(orc.energy())
    assert gpu.status() == 0
    eg, eo = np.array(eg), np.array(eo)
    dev_g = np.max(np.abs(eg / eg[0] - 1.0))
    dev_o = np.max(np.abs(eo / eo[0] - 1.0))
    print("energy deviation over 10000 steps: gpu %.3g oracle %.3g" % (dev_g, dev_o))
    assert eg[0] == pytest.approx(eo[0], rel=1e-5)
    assert dev_g < 0.01
    assert dev_g <= 2.0 * dev_o + 1e-3


@pytest.mark.parametrize("scheme", ["ec_explicit", "ec_implicit"])
def test_stretched_discharge_steps_cleanly_with_sheaths(scheme):
    """The stretched production discharges (cells 0.5x the uniform width at
    the electrodes, 1.5x mid-gap; explicit at 512 cells, direct implicit at
    128 cells and omega_p dt = 2) with a quarter of their particles, for two
    RF periods: clean status, every particle accounted for by the walls and
    the births, electrons depleted next to both electrodes (the sheaths) and
    the bulk density within a factor 2 of the load density."""
    from paper_1310_5284_gb300.sim import Sim
    base = workloads.CFG_WIDE_STRETCHED if scheme == "ec_explicit" else workloads.CFG_IMPLICIT_STRETCHED
    cfg = dict(base, np_init=base["np_init"] // 4)
    period = int(round(1.0 / (cfg["rf_freq"] * cfg["dt"])))
    gpu = Sim(cfg, device="cuda:0")
    gpu.step(period)
    gpu.diag(reset_avg=True)
    gpu.step(period)
    d = gpu.diag()
    assert gpu.status() == 0
    for k in range(2):
        assert d["count"][k] == cfg["np_init"] + d["births"] - sum(d["wall_count"][k])
    prof = gpu.profiles()
    ne, ni = prof["ne"], prof["ni"]
    n = len(ne) - 1
    edge = n // 20
    assert ne[1:edge].mean() < ni[1:edge].mean() and ne[n - edge:n].mean() < ni[n - edge:n].mean()
    assert 0.5 * cfg["n0"] < ne[n // 2] < 2.0 * cfg["n0"]


@pytest.mark.parametrize("scheme,dt,steps", [("ec_explicit", None, 20), ("ec_implicit", 8e-10, 5)])
def test_equal_widths_match_the_uniform_kernel(scheme, dt, steps):
    """The non-uniform modes given cell_width = L/N everywhere against the
    uniform modes, both on the GPU from the same injected state: the node
    charges of the state are identical and after 20 collisionless steps (5
    direct-implicit steps at omega_p dt = 2, as in the oracle comparisons)
    every particle agrees within 1e-5 (of L, of max(|v|, v_th)) or within 4x
    the oracle's own divergence under FP32 rounding over the same steps: the
    two differ only in the order of FP32 roundings (d / h against v dt / dx)."""
    from test_gpu_parity import fp32_sensitivity
    from paper_1310_5284_gb300.sim import Sim
    base = dict(workloads.CFG_SMALL_CCP, np_init=12_800, mcc=False, scheme=scheme, sort_period=8)
    if dt is not None:
        base["dt"] = dt
    n, length = base["n_cells"], base["length"]
    vth = [math.sqrt(E * 2.0 / ME), math.sqrt(E * 0.026 / (39.948 * 1.66053906660e-27))]
    st = [workloads.injected_particles(31 + k, 12_800, n, vth[k]) for k in range(2)]
    out = []
    for cfg in (base, dict(base, cell_width=[length / n] * n)):
        g = Sim(cfg, device="cuda:0")
        for k, sp in enumerate(("e", "i")):
            g.set_particles(sp, dict(st[k], abar=None), next_id=12_800)
        g.init_field(set_abar=True)
        q0 = g.grids()
        g.step(steps)
        assert g.status() == 0
        out.append((q0, {sp: g.get_particles(sp) for sp in ("e", "i")}))
        g.close()
    (qa, pa), (qb, pb) = out
    floor = fp32_sensitivity(base, st, steps)
    assert np.array_equal(qa["rho_q_e"], qb["rho_q_e"]) and np.array_equal(qa["rho_q_i"], qb["rho_q_i"])
    for k, sp in enumerate(("e", "i")):
        a = {key: v[np.argsort(pa[sp]["id"])] for key, v in pa[sp].items() if isinstance(v, np.ndarray)}
        b = {key: v[np.argsort(pb[sp]["id"])] for key, v in pb[sp].items() if isinstance(v, np.ndarray)}
        assert np.array_equal(a["id"], b["id"])
        xa = a["cell"].astype(np.float64) + a["off"]
        xb = b["cell"].astype(np.float64) + b["off"]
        assert np.max(np.abs(xa - xb)) <= max(1e-5 * n, floor[k]["xmax"])
        dv = np.abs(a["vx"].astype(np.float64) - b["vx"]) / np.maximum(np.abs(b["vx"]), vth[k])
        assert dv.max() <= max(1e-5, floor[k]["vmax"]), (sp, dv.max(), floor[k]["vmax"])
