"""Adjoint of the collisionless EC explicit step on the GPU (pic_adj_*).

* The adjoint's forward run is the product step: advanced from the same
  state, every particle is bit-identical to pic_step's (collisionless, frozen
  ions), absorbed particles included.
* Gradients against the FP64 oracle's discrete adjoint on the same state.  The
  GPU differentiates its FP32 trajectory with 16-bit offset quantisation in the
  charge assignment; the bar is 8x the oracle's own change of gradient when its
  initial positions move by the quantisation step (a uniform +-2^-17 cell) and
  its velocities by FP32 rounding, floored at 2e-4.
* dJ/dV0 against central finite differences of the GPU forward run, h = 1e-4
  relative, with the absorbed set unchanged (no event changes).
* The checkpoint period changes nothing but the order of floating-point sums.
* torch.autograd.Function wiring.
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


def spec_for(periodic, n_cells=64, n_particles=8192, nsteps=100, n0=1e15, length=0.01, wpdt=0.2,
             checkpoint_every=20, step0=0, dt=None, bg_density=None):
    dt = dt if dt is not None else wpdt / math.sqrt(n0 * E * E / (EPS0 * ME))
    return dict(periodic=periodic, n_cells=n_cells, n_particles=n_particles, nsteps=nsteps, n0=n0,
                bg_density=n0 if bg_density is None else bg_density, length=length, dt=dt,
                rf_freq=0.0 if periodic else 1.0 / (160 * dt), checkpoint_every=checkpoint_every, step0=step0)


def state_for(spec, seed, te_ev=1.0):
    st = workloads.injected_particles(seed, spec["n_particles"], spec["n_cells"], math.sqrt(E * te_ev / ME),
                                      sorted_cells=True)
    return st


def device_state(st):
    import torch
    return (torch.from_numpy(st["cell"]).cuda(), torch.from_numpy(st["off"]).cuda(),
            torch.from_numpy(st["vx"]).cuda())


def oracle_problem(spec, volt, c_power=1.0, c_flux=0.0):
    w = spec["n0"] * spec["length"] / spec["n_particles"]
    return oracle.adj_problem(spec["n_cells"], spec["periodic"], spec["nsteps"], spec["length"], spec["dt"],
                              rf_freq=spec["rf_freq"], rf_volt=volt, weight=w, bg_density=spec["bg_density"],
                              step0=spec["step0"], c_power=c_power, c_flux=c_flux)


def sim_config(spec, volt):
    return dict(n_cells=spec["n_cells"], periodic=spec["periodic"], length=spec["length"], dt=spec["dt"],
                rf_freq=spec["rf_freq"], rf_volt=volt, n0=spec["n0"], bg_density=spec["bg_density"],
                np_init=spec["n_particles"], mcc=False, ions_mobile=False, sort_period=0,
                capacity=spec["n_particles"], births_capacity=16, eedf_bins=8)


@pytest.mark.parametrize("periodic", [0, 1])
def test_forward_is_the_product_step(periodic):
    from paper_1310_5284_gb300.adjoint import AdjointRun
    from paper_1310_5284_gb300.sim import Sim

    spec = spec_for(periodic, n_particles=5000, nsteps=37, checkpoint_every=8, step0=11)
    volt = 40.0
    st = state_for(spec, 21)
    st["id"] = np.arange(spec["n_particles"], dtype=np.uint32)
    run = AdjointRun(spec)
    run.forward(volt, *device_state(st))
    fin = run.final_state()
    sim = Sim(sim_config(spec, volt))
    sim.set_particles("e", st, next_id=spec["n_particles"])
    sim.set_step(spec["step0"])
    sim.init_field()
    sim.step(spec["nsteps"])
    got = sim.get_particles("e")
    alive = fin["cell"] >= 0
    assert got["id"].size == int(alive.sum())
    if not periodic:
        assert (~alive).sum() > 0  # the case exercises absorption
    ids = got["id"].astype(np.int64)
    for key in ("cell", "off", "vx"):
        assert np.array_equal(fin[key][ids], got[key]), key
    run.close()
    sim.close()


def gradient_bar(spec, st, volt, c_power, c_flux):
    """8x the oracle's gradient change under a quantisation-size move of the
    initial positions and an FP32-rounding move of the velocities."""
    rng = np.random.default_rng(99)
    xi = workloads.xi_of(st)
    vx = st["vx"].astype(np.float64)
    pb = oracle_problem(spec, volt, c_power, c_flux)
    g0 = oracle.adj_gradient(pb, xi, vx)
    xi2 = xi + rng.uniform(-2.0 ** -17, 2.0 ** -17, xi.size)
    if not spec["periodic"]:
        xi2 = np.clip(xi2, 0.0, spec["n_cells"] - 1e-9)
    vx2 = vx * (1.0 + rng.uniform(-2.0 ** -24, 2.0 ** -24, vx.size))
    g1 = oracle.adj_gradient(pb, xi2 % spec["n_cells"] if spec["periodic"] else xi2, vx2)
    dv = np.linalg.norm(g1["dvx0"] - g0["dvx0"]) / np.linalg.norm(g0["dvx0"])
    dV = abs(g1["dV0"] - g0["dV0"]) / max(abs(g0["dV0"]), 1e-300)
    return g0, max(8 * dv, 2e-4), max(8 * dV, 2e-4)


@pytest.mark.parametrize("periodic,c_power,c_flux", [(1, 1.0, 0.0), (1, 0.0, 1e-18), (0, 1.0, 0.0),
                                                     (0, 0.0, 1e-18)])
def test_gradient_matches_oracle(periodic, c_power, c_flux):
    import torch
    from paper_1310_5284_gb300.adjoint import AdjointRun

    spec = spec_for(periodic)
    volt = 0.0 if periodic else 20.0
    st = state_for(spec, 5)
    g0, bar_v, bar_V = gradient_bar(spec, st, volt, c_power, c_flux)
    run = AdjointRun(spec)
    p, g = run.forward(volt, *device_state(st))
    r = oracle.adj_forward(oracle_problem(spec, volt), workloads.xi_of(st), st["vx"].astype(np.float64))
    # objectives: within 1e-3 of themselves or of their natural scales (kinetic
    # energy over the run time, n0 times the mean speed)
    w = spec["n0"] * spec["length"] / spec["n_particles"]
    ke = 0.5 * ME * w * float(np.sum(st["vx"].astype(np.float64) ** 2))
    assert abs(p - r["power"]) <= 1e-3 * abs(r["power"]) + 1e-4 * ke / (spec["nsteps"] * spec["dt"])
    assert abs(g - r["flux"]) <= 1e-3 * abs(r["flux"]) + 1e-4 * spec["n0"] * float(np.abs(st["vx"]).mean())
    g_v, g_x, d_volt = run.backward(c_power, c_flux, want_x0=True)
    torch.cuda.synchronize()
    gv = g_v.cpu().numpy().astype(np.float64)
    alive = run.final_state()["cell"] >= 0
    same = alive == (r["absorbed_at"] < 0)
    assert (~same).sum() <= max(2, spec["n_particles"] // 1000)
    err_v = np.linalg.norm((gv - g0["dvx0"])[same]) / np.linalg.norm(g0["dvx0"][same])
    print("periodic", periodic, "bar_v", bar_v, "err_v", err_v, "dV0", d_volt, g0["dV0"], "bar_V", bar_V)
    assert err_v <= bar_v
    gx = g_x.cpu().numpy().astype(np.float64) * spec["length"] / spec["n_cells"]  # per cell
    err_x = np.linalg.norm((gx - g0["dxi0"])[same]) / np.linalg.norm(g0["dxi0"][same])
    assert err_x <= 4 * bar_v
    if periodic:
        assert d_volt == 0.0
    else:
        assert abs(d_volt - g0["dV0"]) <= bar_V * abs(g0["dV0"])
    run.close()


def test_dV0_matches_finite_differences():
    """A cold, dilute electron cloud in the middle of a driven gap: nothing
    reaches an electrode within the run, so no event can change."""
    from paper_1310_5284_gb300.adjoint import AdjointRun

    spec = spec_for(0, n_particles=65536, nsteps=80, n0=1e12, bg_density=0.4e12, dt=5e-11)
    st = workloads.injected_particles(8, spec["n_particles"], spec["n_cells"], math.sqrt(E * 0.1 / ME),
                                      lo=0.3 * spec["n_cells"], hi=0.7 * spec["n_cells"], sorted_cells=True)
    volt = 1.0
    run = AdjointRun(spec)
    cell, off, vx = device_state(st)
    run.forward(volt, cell, off, vx)
    _, _, d_volt = run.backward(1.0, 0.0)
    h = 1e-4 * volt
    pp, _ = run.forward(volt + h, cell, off, vx)
    ap = run.final_state()["cell"] >= 0
    pm, _ = run.forward(volt - h, cell, off, vx)
    am = run.final_state()["cell"] >= 0
    assert ap.all() and am.all()  # no absorption event at all
    fd = (pp - pm) / (2 * h)
    assert d_volt == pytest.approx(fd, rel=2e-2)
    run.close()


def test_checkpoint_period_only_reorders_sums():
    from paper_1310_5284_gb300.adjoint import AdjointRun

    ref = None
    for C in (20, 1, 7, 100):
        spec = spec_for(0, n_particles=4096, nsteps=60, checkpoint_every=C)
        st = state_for(spec, 4)
        run = AdjointRun(spec)
        p, g = run.forward(15.0, *device_state(st))
        g_v, _, d_volt = run.backward(0.5, 2e-19)
        # a second backward on the same forward run recomputes every segment
        g_v2, _, d_volt2 = run.backward(0.5, 2e-19)
        gv = g_v.cpu().numpy()
        assert np.allclose(g_v2.cpu().numpy(), gv, rtol=1e-5, atol=1e-6 * np.abs(gv).max())
        assert d_volt2 == pytest.approx(d_volt, rel=1e-6)
        if ref is None:
            ref = (p, g, gv, d_volt)
        else:
            assert p == ref[0] and g == ref[1]  # the forward run does not depend on C
            assert np.allclose(gv, ref[2], rtol=1e-5, atol=1e-6 * np.abs(ref[2]).max())
            assert d_volt == pytest.approx(ref[3], rel=1e-6)
        run.close()


def test_autograd_function():
    import torch
    from paper_1310_5284_gb300.adjoint import AdjointRun, ECStepFn

    spec = spec_for(0, n_particles=4096, nsteps=40)
    st = state_for(spec, 6)
    run = AdjointRun(spec)
    cell, off, vx = device_state(st)
    volt = torch.tensor(25.0, dtype=torch.float64, requires_grad=True)
    v0 = vx.clone().requires_grad_(True)
    out = ECStepFn.apply(volt, v0, run, cell, off)
    loss = 2.0 * out[0] - 3e-19 * out[1]
    run.forward(10.0, cell, off, vx)  # another forward run in between: backward must redo its own
    loss.backward()
    run.forward(25.0, cell, off, vx)
    g_v, _, d_volt = run.backward(2.0, -3e-19)
    assert volt.grad.item() == pytest.approx(d_volt, rel=1e-6)
    assert torch.allclose(v0.grad, g_v, rtol=1e-5, atol=1e-6 * float(g_v.abs().max()))
    run.close()


def test_invalid_configurations_are_rejected():
    import ctypes
    from paper_1310_5284_gb300 import _abi
    from paper_1310_5284_gb300.adjoint import make_adj_config

    s = _abi.PicSizes()
    for bad in (dict(n_cells=1), dict(n_cells=2048), dict(n_particles=0), dict(nsteps=0),
                dict(checkpoint_every=0)):
        c = make_adj_config(dict(spec_for(0), **bad))
        assert _abi.lib().pic_adj_required_sizes(ctypes.byref(c), ctypes.byref(s)) < 0
    c = make_adj_config(dict(spec_for(0), n_particles=1 << 29))
    assert _abi.lib().pic_adj_required_sizes(ctypes.byref(c), ctypes.byref(s)) == -4
