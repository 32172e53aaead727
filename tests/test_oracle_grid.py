"""Pins of the oracle's grid operations against what the paper and the
mathematics fix (no GPU): charge assignment Eq. (2), force interpolation
Eq. (3), the energy-conserving property that defines the EC scheme (Sec. 2),
the self-force it introduces (Sec. 1 and Sec. 4), and the field solve."""
import math
from fractions import Fraction

import numpy as np
import pytest
from scipy.interpolate import BSpline

import oracle

EPS0 = 8.8541878128e-12


def cfg(n_cells=8, periodic=False, length=None, **kw):
    c = dict(n_cells=n_cells, periodic=periodic, length=length or float(n_cells), dt=1e-10,
             n0=1.0, np_init=1.0, scheme="ec_explicit")
    c.update(kw)
    return c


def bspline(order):
    """Centred cardinal B-spline of the given order (S_0 = box, S_1 = hat, S_2
    = quadratic) from scipy's Cox-de Boor evaluation."""
    knots = np.arange(order + 2) - (order + 1) / 2.0
    return BSpline.basis_element(knots, extrapolate=False)


def s2_reference(n_cells, xi, periodic):
    """S_2 weights of one particle on all nodes by direct evaluation of the
    quadratic B-spline, with the ghost nodes beyond a wall folded onto it."""
    s2 = bspline(2)
    w = np.zeros(n_cells + 1)
    for g in range(-2, n_cells + 3):
        val = s2(g - xi)
        if np.isnan(val) or val == 0.0:
            continue
        if periodic:
            w[g % n_cells] += val
        else:
            w[min(max(g, 0), n_cells)] += val
    return w


def test_s2_fixed_weights_are_exact_bspline_values():
    # offsets with at most 16 fractional bits are represented exactly by the
    # fixed-point code, so each weight must equal 2^33 * S_2 exactly.
    rng = np.random.default_rng(0)
    s2 = bspline(2)
    for _ in range(200):
        cell = int(rng.integers(1, 7))
        code = int(rng.integers(0, 65536))
        xi = cell + code / 65536.0
        got = oracle.deposit_s2_fixed(cfg(8), [xi])
        for g in range(9):
            val = s2(g - xi) if abs(g - xi) < 1.5 else 0.0
            exact = Fraction(float(val)) * 2 ** 33
            assert exact.denominator == 1, "spline value should be dyadic with 33 bits"
            assert int(got[g]) == exact.numerator


def test_s2_fixed_partition_of_unity_and_fp64_agreement():
    rng = np.random.default_rng(1)
    for periodic in (False, True):
        xi = rng.uniform(0, 16, 5000)
        q = oracle.deposit_s2_fixed(cfg(16, periodic), xi)
        assert q.sum() == len(xi) * 2 ** 33  # every particle assigns exactly one charge
        f = oracle.deposit_s2_fp64(cfg(16, periodic), xi)
        assert abs(f.sum() - len(xi)) < 1e-9
        # quantisation moves each particle by < 2^-16 cell; the S_2 slope is <= 1
        assert np.max(np.abs(q / 2.0 ** 33 - f)) <= len(xi) * 2.0 ** -16


@pytest.mark.parametrize("periodic", [False, True])
def test_s2_fp64_matches_direct_bspline_with_walls(periodic):
    rng = np.random.default_rng(2)
    xs = list(rng.uniform(0, 8, 50)) + [0.0, 0.25, 0.5, 7.5, 7.75, 7.999]
    for xi in xs:
        got = oracle.deposit_s2_fp64(cfg(8, periodic), [xi])
        ref = s2_reference(8, xi, periodic)
        np.testing.assert_allclose(got, ref, atol=1e-14)


def test_s1_fixed_is_linear_weighting():
    h = bspline(1)
    rng = np.random.default_rng(3)
    for periodic in (False, True):
        for _ in range(50):
            cell = int(rng.integers(0, 8))
            code = int(rng.integers(0, 65536))
            xi = cell + code / 65536.0
            got = oracle.deposit_s1_fixed(cfg(8, periodic), [xi]) / 2.0 ** 33
            ref = np.zeros(9)
            for g in range(0, 10):
                v = h(g - xi)
                if not np.isnan(v):
                    ref[g % 8 if periodic else min(g, 8)] += v
            np.testing.assert_allclose(got, ref, atol=1e-15)


def test_quantised_code_uses_fp32_offset_and_rounding_to_next_cell():
    # an FP64 offset that rounds up to 1.0f belongs to the next cell
    xi = 3.0 + (1.0 - 2.0 ** -30)
    q = oracle.deposit_s2_fixed(cfg(8), [xi])
    q_ref = oracle.deposit_s2_fixed(cfg(8), [4.0])
    assert np.array_equal(q, q_ref)


@pytest.mark.parametrize("periodic", [False, True])
def test_ec_force_is_minus_gradient_of_assigned_potential_energy(periodic):
    """The EC scheme is defined by F_p = -dU/dx_p with U = q sum_g S_2(x_g - x_p) phi_g
    (Eq. (2) and Eq. (3) together, Sec. 2); brute-force central differences."""
    n = 8
    c = cfg(n, periodic, length=n * 0.5)
    dx = 0.5
    rng = np.random.default_rng(4)
    phi = rng.normal(size=n + 1)
    if periodic:
        phi[n] = phi[0]
    e_cc, _ = oracle.fields(c, phi)
    h = 1e-6
    for xi in list(rng.uniform(0.01, n - 0.01, 60)) + [0.1, n - 0.1]:
        # keep away from the spline knots where the derivative jumps
        if min(abs(xi - 0.5 - np.round(xi - 0.5)), 1) < 2e-6:
            continue
        up = oracle.deposit_s2_fp64(c, [xi + h]) @ phi
        dn = oracle.deposit_s2_fp64(c, [xi - h]) @ phi
        grad = -(up - dn) / (2 * h * dx)
        assert oracle.gather_ec(c, e_cc, xi) == pytest.approx(grad, rel=1e-7, abs=1e-8)


def _self_force(scheme, xi, n=8):
    """Force on a lone particle from its own field in a periodic box."""
    c = cfg(n, True, length=float(n), scheme=scheme)
    dx = 1.0
    if scheme == "mc_explicit":
        q = oracle.deposit_s1_fixed(c, [xi]) / 2.0 ** 33
    else:
        q = oracle.deposit_s2_fp64(c, [xi])
    rho = q / dx
    phi = oracle.solve_periodic(n, dx, rho)
    phi[n] = phi[0]
    e_cc, e_node = oracle.fields(c, phi)
    if scheme == "mc_explicit":
        return oracle.gather_mc(c, e_node, xi), rho, phi
    return oracle.gather_ec(c, e_cc, xi), rho, phi


def test_self_force_zero_for_mc_and_nonzero_energy_gradient_for_ec():
    """Sec. 1 / Sec. 4: the momentum-conserving scheme has no self-force, the
    EC scheme does.  The EC self-force equals -d/dx of the self energy
    W = (1/2) sum_g (rho_g - <rho>) phi_g dx, by brute-force differences (code offsets
    with 16 fractional bits are exact for the S_1 assignment)."""
    rng = np.random.default_rng(5)
    for xi in rng.uniform(0, 8, 25):
        xi_q = math.floor(xi * 65536) / 65536.0
        f_mc, rho, phi = _self_force("mc_explicit", xi_q)
        scale = np.max(np.abs(phi)) / 1.0  # field scale: potential over one cell
        assert abs(f_mc) < 1e-13 * scale
    seen_nonzero = 0
    for xi in list(rng.uniform(0.6, 7.4, 25)):
        if abs((xi % 1.0) - 0.5) < 1e-3 or abs(xi % 1.0) < 1e-3:
            continue
        f_ec, _, _ = _self_force("ec_explicit", xi)
        h = 1e-5

        def w_self(x):
            _, rho, phi = _self_force("ec_explicit", x)
            # energy of the neutralised system: the uniform background that
            # makes the periodic problem solvable is part of the charge
            return 0.5 * float((rho[:8] - rho[:8].mean()) @ phi[:8])

        grad = -(w_self(xi + h) - w_self(xi - h)) / (2 * h)
        scale = np.max(np.abs(_self_force("ec_explicit", xi)[2]))
        assert f_ec == pytest.approx(grad, rel=1e-5, abs=1e-12 * scale)
        seen_nonzero += abs(f_ec) > 1e-4 * scale
    assert seen_nonzero > 10


@pytest.mark.parametrize("chi0", [0.0, 0.7])
def test_dirichlet_poisson_uniform_charge_closed_form(chi0):
    """Uniform rho0 between a driven and a grounded electrode: the discrete
    solution equals V (1 - x/L) + rho0 x (L - x) / (2 eps0 (1 + chi)) at the nodes
    (the second difference of a quadratic is exact)."""
    n, L, V, rho0 = 50, 0.03, 137.0, 3.2e-3
    dx = L / n
    rho = np.full(n + 1, rho0)
    chi = np.full(n, chi0) if chi0 else None
    phi = oracle.solve_dirichlet(n, dx, rho, V, chi)
    x = np.arange(n + 1) * dx
    ref = V * (1 - x / L) + rho0 * x * (L - x) / (2 * EPS0 * (1 + chi0))
    np.testing.assert_allclose(phi, ref, rtol=1e-11, atol=1e-9)


def test_dirichlet_and_periodic_solves_match_dense_linear_algebra():
    rng = np.random.default_rng(6)
    for n in (2, 3, 7, 16):
        dx = 1e-3
        rho = rng.normal(size=n + 1) * 1e-6
        chi = rng.uniform(0, 3, n)
        V = float(rng.normal() * 10)
        phi = oracle.solve_dirichlet(n, dx, rho, V, chi)
        # dense system for phi_1..phi_{n-1}
        m = n - 1
        A = np.zeros((m, m))
        b = rho[1:n] * dx * dx / EPS0
        for k in range(m):
            g = k + 1
            el, er = 1 + chi[g - 1], 1 + chi[g]
            A[k, k] = el + er
            if k > 0:
                A[k, k - 1] = -el
            if k < m - 1:
                A[k, k + 1] = -er
        b[0] += (1 + chi[0]) * V
        np.testing.assert_allclose(phi[1:n], np.linalg.solve(A, b), rtol=1e-10, atol=1e-12)
        assert phi[0] == V and phi[n] == 0.0
    for n in (4, 9, 32):
        dx = 2e-3
        rho = rng.normal(size=n + 1) * 1e-6
        chi = rng.uniform(0, 2, n)
        phi = oracle.solve_periodic(n, dx, rho, chi)
        r = rho[:n] - rho[:n].mean()
        # cyclic residual of -(d/dx)((1+chi) dphi/dx) = r/eps0 at every node
        res = []
        for g in range(n):
            el, er = 1 + chi[(g - 1) % n], 1 + chi[g]
            lhs = -(er * (phi[(g + 1) % n] - phi[g]) - el * (phi[g] - phi[(g - 1) % n])) / dx ** 2
            res.append(lhs - r[g] / EPS0)
        assert np.max(np.abs(res)) < 1e-6 * np.max(np.abs(r / EPS0))


def test_fields_from_potential():
    n = 6
    phi = np.array([3.0, 1.0, 4.0, 1.0, 5.0, 9.0, 2.0])
    e_cc, e_node = oracle.fields(cfg(n, False, length=3.0), phi)
    dx = 0.5
    np.testing.assert_allclose(e_cc, -(np.diff(phi)) / dx)
    assert e_node[0] == (phi[0] - phi[1]) / dx and e_node[n] == (phi[n - 1] - phi[n]) / dx
    np.testing.assert_allclose(e_node[1:n], (phi[:n - 1] - phi[2:]) / (2 * dx))


def test_gather_zero_field_beyond_electrodes():
    n = 8
    e_cc = np.arange(1.0, n + 1)
    c = cfg(n)
    # at xi = 0 the nearest node is 0, delta = 0: half of the ghost field (0) and half of E_1/2
    assert oracle.gather_ec(c, e_cc, 0.0) == pytest.approx(0.5 * e_cc[0])
    assert oracle.gather_ec(c, e_cc, n - 1e-12) == pytest.approx(0.5 * e_cc[-1], rel=1e-9)
    cp = cfg(n, True)
    assert oracle.gather_ec(cp, e_cc, 0.0) == pytest.approx(0.5 * (e_cc[-1] + e_cc[0]))
