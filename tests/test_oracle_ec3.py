"""Pins of the oracle's m = 3 energy-conserving scheme (no GPU): Eq. (2) with
the cubic B-spline S_3 and Eq. (3) with S_2 from the cell centres, the
"larger m" that Sec. 2 allows.  What fixes it: the B-spline values themselves
(scipy's Cox-de Boor evaluation), a unit charge per particle, the defining EC
property F = -dU/dx (Sec. 2), the self-force it brings (Sec. 1), and total
energy conservation where the momentum-conserving scheme self-heats."""
import math
from fractions import Fraction

import numpy as np
import pytest
from scipy.interpolate import BSpline

import oracle
import workloads

E = 1.602176634e-19
ME = 9.1093837015e-31
EPS0 = 8.8541878128e-12
UNIT3 = 6 * 2 ** 36  # fixed-point charge of one particle, m = 3


def cfg(n_cells=8, periodic=False, length=None, **kw):
    c = dict(n_cells=n_cells, periodic=periodic, length=length or float(n_cells), dt=1e-10,
             n0=1.0, np_init=1.0, scheme="ec3_explicit")
    c.update(kw)
    return c


def bspline(order):
    knots = np.arange(order + 2) - (order + 1) / 2.0
    return BSpline.basis_element(knots, extrapolate=False)


def s3_reference(n_cells, xi, periodic):
    """S_3 weights of one particle on all nodes, ghost nodes folded onto the
    wall nodes (or wrapped)."""
    s3 = bspline(3)
    w = np.zeros(n_cells + 1)
    for g in range(-3, n_cells + 4):
        val = s3(g - xi)
        if np.isnan(val) or val == 0.0:
            continue
        if periodic:
            w[g % n_cells] += val
        else:
            w[min(max(g, 0), n_cells)] += val
    return w


def test_charge_unit():
    assert oracle.charge_unit(cfg()) == UNIT3
    assert oracle.charge_unit(cfg(scheme="ec_explicit")) == 2 ** 33


def test_s3_fixed_weights_are_exact_bspline_values():
    # offsets with 12 fractional bits are held exactly by the code, and
    # 6 * 2^36 S_3 is then an integer (S_3 is a cubic with denominator 6)
    rng = np.random.default_rng(0)
    s3 = bspline(3)
    for _ in range(200):
        cell = int(rng.integers(2, 6))
        code = int(rng.integers(0, 4096))
        xi = cell + code / 4096.0
        got = oracle.deposit_s3_fixed(cfg(8), [xi])
        for g in range(9):
            val = s3(g - xi) if abs(g - xi) < 2.0 else 0.0
            exact = Fraction(float(val)) * UNIT3
            # the FP64 spline value is the rounded cubic: compare to within its rounding
            assert abs(int(got[g]) - exact) <= 2 ** -40 * UNIT3
            # and the integer is the exact rational value of the cubic
            t = Fraction(code, 4096)
            d = abs(Fraction(g) - (cell + t))
            if d < 1:
                ref = (Fraction(2, 3) - d * d + d ** 3 / 2) * UNIT3
            elif d < 2:
                ref = (2 - d) ** 3 / 6 * UNIT3
            else:
                ref = Fraction(0)
            assert ref.denominator == 1 and int(got[g]) == ref.numerator


def test_s3_fixed_partition_of_unity_and_fp64_agreement():
    rng = np.random.default_rng(1)
    for periodic in (False, True):
        xi = rng.uniform(0, 16, 5000)
        q = oracle.deposit_s3_fixed(cfg(16, periodic), xi)
        assert q.sum() == len(xi) * UNIT3  # every particle assigns exactly one charge
        f = oracle.deposit_s3_fp64(cfg(16, periodic), xi)
        assert abs(f.sum() - len(xi)) < 1e-9
        # the 12-bit code moves a particle by < 2^-12 cell; |S_3'| <= 1/2
        assert np.max(np.abs(q / UNIT3 - f)) <= len(xi) * 2.0 ** -13


@pytest.mark.parametrize("periodic", [False, True])
def test_s3_fp64_matches_direct_bspline_with_walls(periodic):
    rng = np.random.default_rng(2)
    xs = list(rng.uniform(0, 8, 50)) + [0.0, 0.25, 0.5, 1.0, 7.0, 7.5, 7.999]
    for xi in xs:
        got = oracle.deposit_s3_fp64(cfg(8, periodic), [xi])
        ref = s3_reference(8, xi, periodic)
        np.testing.assert_allclose(got, ref, atol=1e-14)


def test_s2_gather_from_cell_centres_matches_direct_bspline():
    rng = np.random.default_rng(3)
    s2 = bspline(2)
    for periodic in (False, True):
        c = cfg(8, periodic)
        e_cc = rng.normal(size=8)
        for xi in list(rng.uniform(0, 8, 60)) + [0.0, 0.5, 7.5, 7.999]:
            ref = 0.0
            for cc in range(-2, 11):
                v = s2(xi - (cc + 0.5))
                if np.isnan(v) or v == 0.0:
                    continue
                if periodic:
                    ref += v * e_cc[cc % 8]
                elif 0 <= cc < 8:
                    ref += v * e_cc[cc]  # ghost cells beyond an electrode hold E = 0
            assert oracle.gather_ec3(c, e_cc, xi) == pytest.approx(ref, rel=1e-13, abs=1e-13)


@pytest.mark.parametrize("periodic", [False, True])
def test_ec3_force_is_minus_gradient_of_assigned_potential_energy(periodic):
    """F_p = -dU/dx_p with U = q sum_g S_3(x_g - x_p) phi_g, by central
    differences: the property that makes the scheme energy-conserving."""
    n = 8
    c = cfg(n, periodic, length=n * 0.5)
    dx = 0.5
    rng = np.random.default_rng(4)
    phi = rng.normal(size=n + 1)
    if periodic:
        phi[n] = phi[0]
    e_cc, _ = oracle.fields(c, phi)
    h = 1e-6
    for xi in list(rng.uniform(0.01, n - 0.01, 60)) + [0.1, 0.9, n - 0.1]:
        if abs(xi - round(xi)) < 2e-6:  # knots of S_3 (and of the S_2 gather)
            continue
        up = oracle.deposit_s3_fp64(c, [xi + h]) @ phi
        dn = oracle.deposit_s3_fp64(c, [xi - h]) @ phi
        grad = -(up - dn) / (2 * h * dx)
        assert oracle.gather_ec3(c, e_cc, xi) == pytest.approx(grad, rel=1e-7, abs=1e-8)


def test_ec3_self_force_is_gradient_of_self_energy():
    """A lone particle in a periodic box feels its own field (Sec. 1: the EC
    schemes trade momentum for energy conservation); that force is -dW/dx of
    its self energy W = (1/2) sum_g (rho_g - <rho>) phi_g dx."""
    n = 8

    def solve(x):
        c = cfg(n, True, length=float(n))
        rho = oracle.deposit_s3_fp64(c, [x])
        phi = oracle.solve_periodic(n, 1.0, rho)
        phi[n] = phi[0]
        e_cc, _ = oracle.fields(c, phi)
        return oracle.gather_ec3(c, e_cc, x), rho, phi

    rng = np.random.default_rng(5)
    nonzero = 0
    for xi in rng.uniform(0.6, 7.4, 25):
        if abs(xi - round(xi)) < 1e-3 or abs(xi - round(xi) - 0.5) < 1e-3:
            continue
        f, _, phi = solve(xi)
        h = 1e-5

        def w_self(x):
            _, rho, ph = solve(x)
            return 0.5 * float((rho[:n] - rho[:n].mean()) @ ph[:n])

        grad = -(w_self(xi + h) - w_self(xi - h)) / (2 * h)
        scale = np.max(np.abs(phi))
        assert f == pytest.approx(grad, rel=1e-5, abs=1e-12 * scale)
        nonzero += abs(f) > 1e-5 * scale
    assert nonzero > 10


def test_quasi_neutral_load_has_zero_net_charge_exactly():
    c = dict(workloads.CFG_SMALL_CCP, np_init=3000, scheme="ec3_explicit", quantized=True)
    sim = oracle.Sim(c).load(3000, 3000)
    g = sim.grids()
    assert int(g["rho_q_e"].sum()) == 3000 * UNIT3
    assert int(g["rho_q_i"].sum()) == 3000 * UNIT3


def _thermal_periodic(scheme, wdt, steps, seed=11):
    n0, te = 1e15, 2.0
    lam = math.sqrt(EPS0 * te / (n0 * E))
    n_cells, ppc = 64, 64
    wp = math.sqrt(n0 * E * E / (EPS0 * ME))
    c = workloads.cfg_periodic(n_cells=n_cells, np_e=n_cells * ppc, n0=n0, length=n_cells * 10 * lam,
                               dt=wdt / wp, te_ev=te, scheme=scheme, seed=seed)
    c["quantized"] = False
    sim = oracle.Sim(c).load(n_cells * ppc, 0)
    sim.step(1)
    tot = [sim.energy()]
    for _ in range(steps // 50):
        sim.step(50)
        tot.append(sim.energy())
    return np.array(tot)


def test_ec3_conserves_energy_with_second_order_error():
    """dx = 10 lambda_D, 1000 / omega_p: total energy within 1% at omega_p dt
    = 0.1 and its error grows as dt^2 (ratio 4 for a doubled step), as for
    m = 2 (where the momentum-conserving scheme heats, test_oracle_dynamics)."""
    tot2 = _thermal_periodic("ec3_explicit", 0.2, 5000)
    tot1 = _thermal_periodic("ec3_explicit", 0.1, 10000)
    dev2 = np.max(np.abs(tot2 / tot2[0] - 1.0))
    dev1 = np.max(np.abs(tot1 / tot1[0] - 1.0))
    assert dev1 < 0.01
    assert 3.0 < dev2 / dev1 < 5.0
