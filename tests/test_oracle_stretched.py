"""Pins of the oracle on a non-uniform grid (no GPU): the multi-scale grid of
Sec. 4.  The paper gives no form of Eq. (2)-(3) for unequal cells; the oracle
keeps them in the cell coordinate and takes the force as the x-derivative of
the particle's potential energy, with the Gauss law on the physical nodes.
What fixes it: closed-form potentials the three-point Gauss law reproduces
exactly on any spacing, F = -dU/dx by central differences (Sec. 2's defining
property), free streaming through cells of different widths, the uniform
grid as the special case of equal widths, the density of a uniform load, and
total energy conservation with the second-order error of the uniform grid."""
import math

import numpy as np
import pytest

import oracle
import workloads

E = 1.602176634e-19
ME = 9.1093837015e-31
EPS0 = 8.8541878128e-12


def widths(n, length, beta):
    return np.array(workloads.stretched_widths(n, length, beta))


def test_stretched_widths_follow_the_map():
    h = widths(40, 0.04, 0.6)
    assert h.sum() == pytest.approx(0.04, rel=1e-15)
    # cells (1 - beta) L/N wide at the electrodes and (1 + beta) L/N mid-gap, to O(1/N^2)
    assert h[0] == pytest.approx(0.4 * 0.04 / 40, rel=0.01)
    assert h[19] == pytest.approx(1.6 * 0.04 / 40, rel=0.01)
    assert np.allclose(h, h[::-1], rtol=1e-12)
    assert np.array_equal(widths(8, 1.0, 0.0), np.full(8, 0.125))


def test_locate_inverts_the_node_positions():
    h = widths(33, 0.05, 0.7)
    xn = oracle.grid_nodes(h)
    assert xn[0] == 0.0 and xn[-1] == pytest.approx(0.05, rel=1e-15)
    assert np.allclose(np.diff(xn), h, rtol=1e-12)
    rng = np.random.default_rng(1)
    for x in list(rng.uniform(0.0, 0.05, 300)) + list(xn[:-1]):
        w, c, off = oracle.locate(h, xn, x)
        assert w == 0
        assert c == int(np.searchsorted(xn, x, side="right")) - 1
        assert 0.0 <= off < 1.0
        assert xn[c] + off * h[c] == pytest.approx(x, rel=1e-14, abs=1e-18)
    assert oracle.locate(h, xn, -1e-9)[0] == -1
    assert oracle.locate(h, xn, xn[-1])[0] == 1


@pytest.mark.parametrize("beta", [0.0, 0.5, 0.8])
def test_gauss_law_reproduces_the_parabola_of_uniform_space_charge(beta):
    """Uniform space charge rho0 between the driven and the grounded
    electrode: phi = V (1 - x/L) + rho0 x (L - x) / (2 eps0).  The three-point
    Gauss law is exact for a quadratic on any spacing when node g carries
    rho0 (h_{g-1} + h_g) / 2."""
    n, length, rho0, v = 24, 0.03, 3.0e-6, 150.0
    h = widths(n, length, beta)
    xn = oracle.grid_nodes(h)
    q = np.zeros(n + 1)
    q[1:n] = rho0 * 0.5 * (h[:-1] + h[1:])
    phi = oracle.solve_dirichlet_h(h, q, v)
    exact = v * (1.0 - xn / length) + rho0 * xn * (length - xn) / (2.0 * EPS0)
    assert np.allclose(phi, exact, rtol=1e-11, atol=1e-11 * np.abs(exact).max())


def test_periodic_solve_spreads_the_net_charge_by_node_length():
    """One charge Q on node 0 of a periodic box: the neutralising charge is
    -Q/L per metre, spread as (h_{g-1} + h_g)/2 over the nodes, and the
    potential with phi_0 = 0 is Q (x^2/L - x) / (2 eps0), exact at the nodes."""
    n, length, qq = 20, 0.02, 4.0e-9
    h = widths(n, length, 0.6)
    xn = oracle.grid_nodes(h)
    q = np.zeros(n + 1)
    q[0] = qq
    phi = oracle.solve_periodic_h(h, q)
    exact = qq * (xn ** 2 / length - xn) / (2.0 * EPS0)
    assert np.allclose(phi[:n], exact[:n], rtol=1e-11, atol=1e-11 * np.abs(exact).max())


def _potential_energy(c, phi, xn, h, x, m=2):
    """q = 1: U(x) = sum_g phi_g S_m(xi(x) - g), ghost nodes folded or wrapped."""
    w, cell, off = oracle.locate(h, xn, x)
    assert w == 0
    dep = oracle.deposit_s2_fp64 if m == 2 else oracle.deposit_s3_fp64
    return float(dep(c, [cell + off]) @ phi)


@pytest.mark.parametrize("periodic,m", [(False, 2), (True, 2), (False, 3), (True, 3)])
def test_force_is_minus_gradient_of_the_assigned_potential_energy(periodic, m):
    """The gathered field is -dU/dx for a unit charge, by central differences
    in the physical coordinate, on a grid whose cells differ by up to 5x
    (m = 2: S_2 assignment, S_1 interpolation; m = 3: S_3 and S_2)."""
    n, length = 12, 0.012
    h = widths(n, length, 0.65)
    xn = oracle.grid_nodes(h)
    c = dict(n_cells=n, periodic=periodic, length=length, dt=1e-10, n0=1.0, np_init=1.0,
             scheme="ec_explicit" if m == 2 else "ec3_explicit", cell_width=h)
    gather = oracle.gather_ec_h if m == 2 else oracle.gather_ec3_h
    rng = np.random.default_rng(3)
    phi = rng.normal(size=n + 1) * 10.0
    if periodic:
        phi[n] = phi[0]
    u = np.array([phi[k] - (phi[0] if periodic and k + 1 == n else phi[k + 1]) for k in range(n)])
    d = 1e-9
    tested = 0
    for x in rng.uniform(0.0, length, 200):
        w, cell, off = oracle.locate(h, xn, x)
        if min(off, 1.0 - off) * h[cell] < 10 * d:  # the map's kinks at the nodes
            continue
        grad = -(_potential_energy(c, phi, xn, h, x + d, m) - _potential_energy(c, phi, xn, h, x - d, m)) / (2 * d)
        assert gather(c, u, cell + off) == pytest.approx(grad, rel=1e-6, abs=1e-6 * np.abs(u).max() / h.min())
        tested += 1
    assert tested > 150


def _free_streaming_cfg(n=16, beta=0.7, periodic=True, scheme="ec_explicit"):
    length = 0.016
    c = dict(n_cells=n, periodic=periodic, length=length, dt=1e-9, n0=1e-6, np_init=4.0,
             scheme=scheme, mcc=False, ions_mobile=True, quantized=False, rf_volt=0.0,
             cell_width=widths(n, length, beta), te_ev=1.0, ti_ev=0.026)
    return c


@pytest.mark.parametrize("scheme", ["ec_explicit", "ec_implicit"])
def test_free_streaming_crosses_cells_of_different_width(scheme):
    """With a vanishing weight the field is negligible, so x(t) = x0 + v t,
    wrapped in the periodic box; velocities cross up to several cells a step
    (the direct-implicit push: predictor and corrector moves alike)."""
    c = _free_streaming_cfg(scheme=scheme)
    h, xn, length = np.asarray(c["cell_width"]), oracle.grid_nodes(c["cell_width"]), c["length"]
    x0 = np.array([0.0005, 0.004, 0.0101, 0.0159])
    v = np.array([3.0e5, -2.2e6, 4.1e6, -7.0e5])
    xi0 = []
    for x in x0:
        _, cell, off = oracle.locate(h, xn, x)
        xi0.append(cell + off)
    sim = oracle.Sim(c, cap_e=8, cap_i=8)
    sim.set_species(0, xi0, v, np.zeros(4), np.zeros(4), np.arange(4))
    sim.set_species(1, xi0, np.zeros(4), np.zeros(4), np.zeros(4), np.arange(4))
    sim.init_field()
    steps = 25
    sim.step(steps)
    got = sim.get_species(0)
    for k in range(4):
        xe = (x0[k] + v[k] * steps * c["dt"]) % length
        cell = int(math.floor(got["xi"][k]))
        xg = xn[cell] + (got["xi"][k] - cell) * h[cell]
        assert xg == pytest.approx(xe, abs=1e-12 * length)
        assert got["vx"][k] == pytest.approx(v[k], rel=1e-9)


def test_free_streaming_is_absorbed_at_the_electrodes():
    c = _free_streaming_cfg(periodic=False)
    h, xn = np.asarray(c["cell_width"]), oracle.grid_nodes(c["cell_width"])
    sim = oracle.Sim(c, cap_e=8, cap_i=8)
    _, c0, o0 = oracle.locate(h, xn, 0.001)
    _, c1, o1 = oracle.locate(h, xn, 0.015)
    sim.set_species(0, [c0 + o0, c1 + o1], [-2.0e5, 2.0e5], [0.0, 0.0], [0.0, 0.0], [0, 1])
    sim.set_species(1, [c0 + o0, c1 + o1], [0.0, 0.0], [0.0, 0.0], [0.0, 0.0], [0, 1])
    sim.init_field()
    sim.step(4)  # 0.8 mm: both still inside
    assert sim.count(0) == 2
    sim.step(2)  # 1.2 mm: both past their electrode
    d = sim.diag()
    assert sim.count(0) == 0 and d["wall_count"][0] == [1, 1]


@pytest.mark.parametrize("scheme", ["ec_explicit", "ec3_explicit"])
def test_equal_widths_reproduce_the_uniform_scheme(scheme):
    """cell_width = L/N everywhere is the uniform grid: the same run (MCC
    off, FP64 weights) through both code paths for 30 steps."""
    base = dict(workloads.CFG_SMALL_CCP, mcc=False, quantized=False, scheme=scheme)
    n, length = base["n_cells"], base["length"]
    stretched = dict(base, cell_width=[length / n] * n)
    vth = math.sqrt(E * 2.0 / ME)
    st = workloads.injected_particles(21, 3000, n, vth)
    xi = workloads.xi_of(st)
    sims = []
    for c in (base, stretched):
        s = oracle.Sim(c, cap_e=4096, cap_i=4096)
        s.set_species(0, xi, st["vx"], st["vy"], st["vz"], st["id"])
        s.set_species(1, xi, 0.01 * st["vx"], st["vy"], st["vz"], st["id"])
        s.init_field()
        s.step(30)
        sims.append(s)
    a, b = sims[0].get_species(0), sims[1].get_species(0)
    assert sims[0].count(0) == sims[1].count(0)
    assert np.array_equal(a["id"], b["id"])
    assert np.allclose(a["xi"], b["xi"], rtol=0, atol=1e-9)
    assert np.allclose(a["vx"], b["vx"], rtol=1e-8, atol=1e-6)
    ga, gb = sims[0].grids(), sims[1].grids()
    assert np.allclose(ga["phi"], gb["phi"], rtol=1e-7, atol=1e-9 * np.abs(ga["phi"]).max())
    assert sims[1].diag()["field_energy"] == pytest.approx(sims[0].diag()["field_energy"], rel=1e-6)


def test_uniform_load_gives_the_load_density_at_every_node():
    """The load is uniform in x: a node's time-averaged density (its charge
    over (h_{g-1} + h_g)/2) is n0 wherever the cells are fine or coarse."""
    c = dict(workloads.cfg_periodic_stretched(n_cells=32, np_sp=200000, beta=0.6), quantized=True)
    sim = oracle.Sim(c).load(200000, 200000)
    got = sim.get_species(0)
    assert np.all((got["xi"] >= 0) & (got["xi"] < 32))
    off = got["xi"] - np.floor(got["xi"])
    assert np.array_equal(off, off.astype(np.float32).astype(np.float64))  # FP32 offsets
    h = np.asarray(c["cell_width"])
    counts = np.bincount(np.floor(got["xi"]).astype(int), minlength=32)
    expect = 200000 * h / h.sum()
    chi2 = float(np.sum((counts - expect) ** 2 / expect))
    assert chi2 < 32 + 5 * math.sqrt(64)  # 31 degrees of freedom
    sim.step(1)
    ne = sim.averages()["ne"][:32]
    assert np.allclose(ne, c["n0"], rtol=0.05)


def test_other_schemes_are_refused_on_a_non_uniform_grid():
    for scheme in ("mc_explicit", "mc_implicit"):
        with pytest.raises(ValueError):
            oracle.Sim(dict(workloads.cfg_periodic_stretched(), scheme=scheme))
    with pytest.raises(ValueError):
        oracle.Sim(dict(workloads.cfg_periodic_stretched(), ions_mobile=False))


@pytest.mark.parametrize("beta", [0.0, 0.5])
def test_modified_poisson_is_the_series_capacitor_in_vacuum(beta):
    """No charge, a susceptibility that varies from cell to cell: D = (1 +
    chi_c) E_c is the same in every cell and sum_c h_c E_c = V, so
    D = V / sum_c h_c / (1 + chi_c) and phi_g = V - D sum_{c<g} h_c / (1 + chi_c)."""
    n, length, v = 30, 0.03, 120.0
    h = widths(n, length, beta)
    chi = np.random.default_rng(8).uniform(0.0, 5.0, n)
    phi = oracle.solve_dirichlet_h(h, np.zeros(n + 1), v, chi=chi)
    d = v / np.sum(h / (1.0 + chi))
    exact = v - d * np.concatenate([[0.0], np.cumsum(h / (1.0 + chi))])
    assert np.allclose(phi, exact, rtol=1e-12, atol=1e-12 * v)


def test_modified_poisson_with_uniform_chi_scales_the_parabola():
    """Uniform space charge and a uniform susceptibility: the parabola of the
    plain Gauss law divided by 1 + chi, on any spacing."""
    n, length, rho0, v, chi0 = 24, 0.03, 3.0e-6, 150.0, 2.5
    h = widths(n, length, 0.7)
    xn = oracle.grid_nodes(h)
    q = np.zeros(n + 1)
    q[1:n] = rho0 * 0.5 * (h[:-1] + h[1:])
    phi = oracle.solve_dirichlet_h(h, q, v, chi=np.full(n, chi0))
    exact = v * (1.0 - xn / length) + rho0 * xn * (length - xn) / (2.0 * EPS0 * (1.0 + chi0))
    assert np.allclose(phi, exact, rtol=1e-11, atol=1e-11 * np.abs(exact).max())


def test_susceptibility_of_a_uniform_plasma_is_the_same_in_every_cell():
    """The direct-implicit susceptibility is (omega_p dt)^2 / 2 summed over
    the species for a uniform density: on a stretched grid a uniform load
    puts counts in proportion to the cell widths, and every cell's chi must
    still come out at that value (within the count noise, 2 % here)."""
    n0, te, dt = 1e15, 2.0, 2e-10
    c = workloads.cfg_periodic_stretched(n_cells=64, np_sp=400_000, n0=n0, length=0.05, dt=dt, te_ev=te, beta=0.6)
    c.update(scheme="ec_implicit", quantized=True)
    sim = oracle.Sim(c).load(400_000, 400_000)
    sim.step(1)
    chi = sim.grids()["chi"]
    mi = c["ion_mass_amu"] * 1.66053906660e-27
    expect = 0.5 * dt * dt * n0 * E * E / EPS0 * (1.0 / ME + 1.0 / mi)
    assert np.allclose(chi, expect, rtol=0.06), (chi.min() / expect, chi.max() / expect)
    assert abs(chi.mean() / expect - 1.0) < 0.01


def test_equal_widths_reproduce_the_uniform_implicit_scheme():
    """The direct-implicit push (Sec. 2 scheme (4)) with cell_width = L/N:
    predictor, susceptibility, modified Poisson and corrector as on the
    uniform grid, 30 steps at omega_p dt = 2 (MCC off, FP64 weights)."""
    base = dict(workloads.CFG_IMPLICIT, n_cells=64, np_init=6000, mcc=False, quantized=False)
    n, length = base["n_cells"], base["length"]
    stretched = dict(base, cell_width=[length / n] * n)
    vth = math.sqrt(E * 2.0 / ME)
    st = workloads.injected_particles(23, 6000, n, vth)
    xi = workloads.xi_of(st)
    sims = []
    for c in (base, stretched):
        s = oracle.Sim(c, cap_e=8192, cap_i=8192)
        s.set_species(0, xi, st["vx"], st["vy"], st["vz"], st["id"])
        s.set_species(1, xi, 0.01 * st["vx"], st["vy"], st["vz"], st["id"])
        s.init_field()
        s.step(30)
        sims.append(s)
    a, b = sims[0].get_species(0), sims[1].get_species(0)
    assert sims[0].count(0) == sims[1].count(0)
    assert np.allclose(a["xi"], b["xi"], rtol=0, atol=1e-8)
    assert np.allclose(a["vx"], b["vx"], rtol=1e-7, atol=1e-5)
    assert np.allclose(a["abar"], b["abar"], rtol=1e-6, atol=1e-6 * np.abs(a["abar"]).max())
    ga, gb = sims[0].grids(), sims[1].grids()
    assert np.allclose(ga["chi"], gb["chi"], rtol=1e-12)
    assert np.allclose(ga["phi"], gb["phi"], rtol=1e-7, atol=1e-8 * np.abs(ga["phi"]).max())


def test_implicit_on_stretched_cells_follows_the_uniform_grid():
    """omega_p dt = 2 (beyond the explicit limit of Eq. (1)) with cells 5 to
    15 Debye lengths: the direct-implicit push damps the load's charge
    fluctuations and cools the plasma (three quarters of the total energy
    go in 1000 steps, on the uniform grid as well); the stretched grid's
    energy history stays within 5 % of the total of the uniform grid's of
    the same mean width (2.2 % measured)."""
    out = []
    for beta in (0.0, 0.5):
        n0, te = 1e15, 2.0
        lam = math.sqrt(EPS0 * te / (n0 * E))
        wp = math.sqrt(n0 * E * E / (EPS0 * ME))
        c = workloads.cfg_periodic_stretched(n_cells=64, np_sp=64 * 64, n0=n0, length=64 * 10 * lam,
                                             dt=2.0 / wp, te_ev=te, beta=beta)
        c.update(scheme="ec_implicit", quantized=False)
        sim = oracle.Sim(c).load(64 * 64, 64 * 64)
        sim.step(1)
        tot = [sim.energy()]
        for _ in range(10):
            sim.step(100)
            tot.append(sim.energy())
        out.append(np.array(tot) / tot[0] - 1.0)
    uni, st = out
    assert uni[-1] < -0.5 and st[-1] < -0.5
    assert np.max(np.abs(st - uni)) < 0.05


def _thermal(wdt, steps, beta=0.5, scheme="ec_explicit"):
    n0, te = 1e15, 2.0
    lam = math.sqrt(EPS0 * te / (n0 * E))
    n_cells, ppc = 64, 64
    wp = math.sqrt(n0 * E * E / (EPS0 * ME))
    c = workloads.cfg_periodic_stretched(n_cells=n_cells, np_sp=n_cells * ppc, n0=n0,
                                         length=n_cells * 10 * lam, dt=wdt / wp, te_ev=te, beta=beta)
    c.update(quantized=False, scheme=scheme)
    sim = oracle.Sim(c).load(n_cells * ppc, n_cells * ppc)
    sim.step(1)
    tot = [sim.energy()]
    for _ in range(steps // 50):
        sim.step(50)
        tot.append(sim.energy())
    return np.array(tot)


@pytest.mark.parametrize("scheme", ["ec_explicit", "ec3_explicit"])
def test_stretched_grid_conserves_energy_with_second_order_error(scheme):
    """Mean dx = 10 lambda_D, cells from 5 to 15 lambda_D, 1000 / omega_p:
    total energy within 1% at omega_p dt = 0.1 and the error grows as dt^2
    (ratio 4 for a doubled step), as on the uniform grid (m = 2 and 3)."""
    tot2 = _thermal(0.2, 5000, scheme=scheme)
    tot1 = _thermal(0.1, 10000, scheme=scheme)
    dev2 = np.max(np.abs(tot2 / tot2[0] - 1.0))
    dev1 = np.max(np.abs(tot1 / tot1[0] - 1.0))
    assert dev1 < 0.01
    assert 3.0 < dev2 / dev1 < 5.0
