"""Pins of the oracle's collisionless EC run and its discrete adjoint.

The adjoint is checked against things other than itself: central finite
differences of the oracle's forward run (small steps, so that no particle
crosses a spline kink or changes its absorption step), a single test particle
in the uniform field of an empty gap whose objective is an explicit quadratic
in the voltage and the initial velocity, the leapfrog energy identity
q E vbar = m (v+^2 - v-^2) / (2 dt) for the absorbed power, and linearity in
the objective weights.
"""
import numpy as np
import pytest

import oracle

E = 1.602176634e-19
ME = 9.1093837015e-31
EPS0 = 8.8541878128e-12


def plasma_case(periodic, n_cells=32, npart=512, steps=50, n0=1e15, length=0.01, volt=0.5, seed=1,
                c_power=1.0, c_flux=0.0):
    rng = np.random.default_rng(seed)
    dt = 0.2 / np.sqrt(n0 * E * E / (EPS0 * ME))
    pb = oracle.adj_problem(n_cells, periodic, steps, length, dt, rf_freq=2.7e8, rf_volt=volt,
                            weight=n0 * length / npart, bg_density=n0, step0=3, c_power=c_power,
                            c_flux=c_flux)
    xi = rng.uniform(0.0, n_cells, npart) if periodic else rng.uniform(0.3 * n_cells, 0.7 * n_cells, npart)
    vx = rng.normal(0.0, 0.3 * np.sqrt(2 * E / ME), npart)
    return pb, xi, vx


def objective(pb, xi, vx, volt=None):
    q = oracle.adj_problem(pb.n_cells, pb.periodic, pb.nsteps, pb.length, pb.dt, pb.rf_freq,
                           pb.rf_volt if volt is None else volt, pb.weight, pb.bg_density, pb.step0)
    r = oracle.adj_forward(q, xi, vx)
    return pb.c_power * r["power"] + pb.c_flux * r["flux"], r["absorbed_at"]


@pytest.mark.parametrize("periodic", [1, 0])
@pytest.mark.parametrize("weights", [(1.0, 0.0), (0.0, 1.0)])
def test_directional_derivatives_match_finite_differences(periodic, weights):
    pb, xi, vx = plasma_case(periodic, c_power=weights[0], c_flux=weights[1])
    g = oracle.adj_gradient(pb, xi, vx)
    j0, ab0 = objective(pb, xi, vx)
    assert g["J"] == pytest.approx(j0, rel=1e-14)
    rng = np.random.default_rng(7)
    h = 1e-5
    dv = rng.normal(size=xi.size) * 1e3                 # m/s
    dxi = rng.normal(size=xi.size) * 1e-3               # cells
    jp, abp = objective(pb, xi, vx + h * dv)
    jm, abm = objective(pb, xi, vx - h * dv)
    assert np.array_equal(abp, ab0) and np.array_equal(abm, ab0)  # no event changed
    fd_v = (jp - jm) / (2 * h)
    assert g["dvx0"] @ dv == pytest.approx(fd_v, rel=1e-5)
    jp, _ = objective(pb, xi + h * dxi, vx)
    jm, _ = objective(pb, xi - h * dxi, vx)
    assert g["dxi0"] @ dxi == pytest.approx((jp - jm) / (2 * h), rel=1e-5)
    if not periodic:
        hv = 1e-4 * pb.rf_volt
        jp, abp = objective(pb, xi, vx, pb.rf_volt + hv)
        jm, abm = objective(pb, xi, vx, pb.rf_volt - hv)
        assert np.array_equal(abp, ab0) and np.array_equal(abm, ab0)
        assert g["dV0"] == pytest.approx((jp - jm) / (2 * hv), rel=1e-5)


def test_single_components_match_finite_differences():
    pb, xi, vx = plasma_case(1, npart=128, steps=40, c_power=0.3, c_flux=2e-17)
    g = oracle.adj_gradient(pb, xi, vx)
    for k in (0, 17, 99):
        for h in (1e-2,):
            e = np.zeros(xi.size)
            e[k] = h
            fd = (objective(pb, xi, vx + e)[0] - objective(pb, xi, vx - e)[0]) / (2 * h)
            assert g["dvx0"][k] == pytest.approx(fd, rel=1e-4, abs=1e-9 * np.abs(g["dvx0"]).max())


def test_test_particle_in_uniform_field_closed_form():
    """One electron of negligible weight in an empty gap: E = V(t_n)/L everywhere
    inside, so v^{n+1/2} = v0 + (q/m) dt sum_{k<=n} V0 s_k / L and the time-averaged
    power is an explicit quadratic in (V0, v0)."""
    n_cells, length, steps, f = 16, 0.02, 30, 13.56e6
    dt = 1.0 / (400 * f)
    volt, v0 = 3.0, 2.0e4
    pb = oracle.adj_problem(n_cells, 0, steps, length, dt, rf_freq=f, rf_volt=volt, weight=1e-12,
                            bg_density=0.0, step0=5, c_power=1.0)
    xi = np.array([0.5 * n_cells])
    g = oracle.adj_gradient(pb, xi, np.array([v0]))
    q, qm = -E, -E / ME
    s = np.sin(2 * np.pi * f * dt * (pb.step0 + np.arange(steps)))
    w = pb.weight
    # v_half[n] = v^{n+1/2} = v0 + a V0 C_n, C_n = sum_{k<=n} s_k, a = qm dt / L
    a = qm * dt / length
    C = np.cumsum(s)
    Cm = np.concatenate([[0.0], C[:-1]])
    # P^n = q w (V0 s_n / L) (v^{n-1/2} + v^{n+1/2}) / 2
    vbar_0 = v0 * np.ones(steps)                         # V0-independent part of vbar
    vbar_1 = a * 0.5 * (C + Cm)                          # coefficient of V0 in vbar
    J = np.mean(q * w * s / length * (volt * vbar_0 + volt * volt * vbar_1))
    dJ_dV0 = np.mean(q * w * s / length * (vbar_0 + 2 * volt * vbar_1))
    dJ_dv0 = np.mean(q * w * s / length * volt)
    # the particle must not have reached a ghost half-cell
    r = oracle.adj_forward(pb, xi, np.array([v0]))
    assert r["absorbed_at"][0] == -1 and 1.0 < r["xi"][0] < n_cells - 1
    assert g["J"] == pytest.approx(J, rel=1e-9)
    assert g["dV0"] == pytest.approx(dJ_dV0, rel=1e-9)
    assert g["dvx0"][0] == pytest.approx(dJ_dv0, rel=1e-9)


def test_power_is_the_kinetic_energy_change():
    """Leapfrog: q E_p vbar = m (v+^2 - v-^2)/(2 dt), so in a periodic box the
    time-averaged power is the kinetic-energy change over the run."""
    pb, xi, vx = plasma_case(1, steps=60)
    r = oracle.adj_forward(pb, xi, vx)
    dke = 0.5 * ME * pb.weight * (np.sum(r["vx"] ** 2) - np.sum(vx ** 2))
    assert r["power"] == pytest.approx(dke / (pb.nsteps * pb.dt), rel=1e-9)


def test_gradient_is_linear_in_the_objective_weights():
    pb, xi, vx = plasma_case(0, npart=256, steps=30)
    out = {}
    for cp, cg in ((1.0, 0.0), (0.0, 1.0), (2.0, -3e-17)):
        pb.c_power, pb.c_flux = cp, cg
        out[(cp, cg)] = oracle.adj_gradient(pb, xi, vx)
    a, b, c = out[(1.0, 0.0)], out[(0.0, 1.0)], out[(2.0, -3e-17)]
    np.testing.assert_allclose(c["dvx0"], 2.0 * a["dvx0"] - 3e-17 * b["dvx0"], rtol=1e-9,
                               atol=1e-12 * np.abs(c["dvx0"]).max())
    assert c["dV0"] == pytest.approx(2.0 * a["dV0"] - 3e-17 * b["dV0"], rel=1e-9)
