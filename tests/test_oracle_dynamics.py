"""Pins of the oracle's time stepping against closed forms and against the
numbers the paper prints (no GPU).

* Sec. 3 prints, for the converged 800-cell benchmark, n ~ 5.2e16 m^-3,
  lambda_D ~ 3.3e-5 m, dx ~ 1.4 lambda_D and omega_p dt ~ 0.2 at dt = 1.5e-11 s.
* Eq. (1): the leapfrog push is stable only for omega_p dt < 2.
* Cold Langmuir oscillation: leapfrog frequency (2/dt) asin(omega_p dt / 2).
* Cold two-stream instability: gamma^2 = -(a^2 + wb^2 - wb sqrt(wb^2 + 4 a^2)), a = k v0.
* Sec. 1: the EC scheme conserves total energy where the momentum-conserving
  scheme self-heats (dx >> lambda_D).
* Sec. 2 scheme (4), direct implicit (D1 form): a cold oscillation follows the
  recurrence whose characteristic polynomial is (z-1)^2 (2z-1) + (omega dt)^2 z^3.
"""
import math

import numpy as np
import pytest

import oracle
import workloads

E = 1.602176634e-19
ME = 9.1093837015e-31
EPS0 = 8.8541878128e-12


def omega_p(n):
    return math.sqrt(n * E * E / (EPS0 * ME))


def cold_plasma(n_cells, ppc, n0, dt, amp, scheme="ec_explicit", length=None, quantized=False,
                beams=None):
    """Periodic cold electron plasma on a frozen ion background, quiet start,
    displaced by amp * sin(2 pi x / L) (cells).  beams=(v0,) gives two cold
    counter-streaming beams of half the density each."""
    n_cells = int(n_cells)
    length = length if length is not None else n_cells * 1e-3
    nb = 2 if beams else 1
    n_per = n_cells * ppc
    xs, vs = [], []
    for b in range(nb):
        xi0 = (np.arange(n_per) + 0.5) / ppc
        xi = xi0 + amp * np.sin(2 * np.pi * xi0 / n_cells)
        xs.append(np.mod(xi, n_cells))
        vs.append(np.full(n_per, 0.0 if not beams else (beams[0] if b == 0 else -beams[0])))
    xi = np.concatenate(xs)
    vx = np.concatenate(vs)
    cfg = workloads.cfg_periodic(n_cells=n_cells, np_e=len(xi), n0=n0, length=length, dt=dt,
                                 scheme=scheme)
    cfg["quantized"] = quantized
    sim = oracle.Sim(cfg, cap_e=len(xi) + 16, cap_i=16)
    z = np.zeros_like(xi)
    sim.set_species("e", xi, vx, z, z, np.arange(len(xi), dtype=np.uint32))
    sim.set_species("i", [], [], [], [], np.zeros(0, dtype=np.uint32), next_id=0)
    sim.init_field()
    return sim, cfg


def mode1(sim, n_cells):
    e = sim.grids()["e_cc"]
    xc = (np.arange(n_cells) + 0.5) / n_cells
    return complex(np.sum(e * np.sin(2 * np.pi * xc)), np.sum(e * np.cos(2 * np.pi * xc)))


def run_series(sim, n_cells, steps):
    a = [mode1(sim, n_cells)]
    for _ in range(steps):
        sim.step(1)
        a.append(mode1(sim, n_cells))
    return np.array(a)


def zero_crossing_frequency(series, dt):
    s = np.real(series)
    idx = np.where(np.sign(s[:-1]) * np.sign(s[1:]) < 0)[0]
    t = [(i + s[i] / (s[i] - s[i + 1])) * dt for i in idx]
    half_periods = len(t) - 1
    return math.pi * half_periods / (t[-1] - t[0])


def test_langmuir_frequency_and_paper_constants():
    """omega_p from a cold oscillation at the paper's converged density and time
    step reproduces the printed omega_p dt ~ 0.2 and lambda_D ~ 3.3e-5 m, and
    the oscillation runs at the leapfrog frequency."""
    n0, dt, n_cells = 5.2e16, 1.5e-11, 64
    dx = 0.04 / 800  # the paper's 4 cm gap on 800 cells
    sim, cfg = cold_plasma(n_cells, 16, n0, dt, 0.02, length=n_cells * dx)
    a = run_series(sim, n_cells, 800)
    w_meas = zero_crossing_frequency(a, dt)
    w_leap = 2.0 / dt * math.asin(omega_p(n0) * dt / 2.0)
    assert w_meas == pytest.approx(w_leap, rel=1e-2)
    wp = 2.0 / dt * math.sin(w_meas * dt / 2.0)  # plasma frequency the oracle realises
    assert round(wp * dt, 1) == 0.2
    vth_1ev = oracle.derive(dict(cfg, te_ev=1.0))["vth"][0]
    lam = vth_1ev / wp
    assert float("%.2g" % lam) == 3.3e-5
    assert dx / lam == pytest.approx(1.4, rel=0.1)


def test_leapfrog_stability_limit_eq1():
    n_cells, n0 = 32, 1e15
    wp = omega_p(n0)
    for wdt, stable in ((1.9, True), (2.2, False)):
        sim, _ = cold_plasma(n_cells, 16, n0, wdt / wp, 1e-3)
        a = np.abs(run_series(sim, n_cells, 14))
        if stable:
            assert a.max() < 5 * a[0]
        else:
            assert a[-1] > 1e3 * a[0]


def test_two_stream_growth_rate():
    n_cells, n0 = 64, 1e15
    L = 0.064
    wp = omega_p(n0)
    wb = wp / math.sqrt(2.0)
    k = 2 * math.pi / L
    v0 = math.sqrt(3.0) / 2.0 * wb / k  # fastest-growing beam speed for mode 1
    dt = 0.05 / wp
    sim, _ = cold_plasma(n_cells, 64, n0, dt, 1e-4, length=L, beams=(v0,))
    a = np.abs(run_series(sim, n_cells, 620))
    la = np.log(a)
    # linear phase: from 3 to 7 e-folds above the seed
    i0 = np.argmax(la > la[0] + 3.0)
    i1 = np.argmax(la > la[0] + 7.0)
    assert i1 > i0 + 50
    slope = np.polyfit(np.arange(i0, i1) * dt, la[i0:i1], 1)[0]
    a_ = k * v0
    gamma = math.sqrt(-(a_ ** 2 + wb ** 2 - wb * math.sqrt(wb ** 2 + 4 * a_ ** 2)))
    assert gamma == pytest.approx(wb / 2.0, rel=1e-12)
    assert slope == pytest.approx(gamma, rel=0.05)


def _thermal_periodic(scheme, wdt, steps, seed=11):
    """Collisionless thermal plasma at dx = 10 Debye lengths."""
    n0, te = 1e15, 2.0
    lam = math.sqrt(EPS0 * te / (n0 * E))
    n_cells, ppc = 64, 64
    dx = 10 * lam
    wp = omega_p(n0)
    cfg = workloads.cfg_periodic(n_cells=n_cells, np_e=n_cells * ppc, n0=n0,
                                 length=n_cells * dx, dt=wdt / wp, te_ev=te, scheme=scheme,
                                 seed=seed)
    cfg["quantized"] = False
    sim = oracle.Sim(cfg).load(n_cells * ppc, 0)
    sim.step(1)
    tot, ke = [sim.energy()], []
    d = sim.diag()
    ke.append(d["ke_x"][0] + d["ke_perp"][0])
    for _ in range(steps // 50):
        sim.step(50)
        d = sim.diag()
        tot.append(sim.energy())
        ke.append(d["ke_x"][0] + d["ke_perp"][0])
    return np.array(tot), np.array(ke)


def test_ec_conserves_energy_where_mc_self_heats():
    """Over 1000 / omega_p at dx = 10 lambda_D the EC total energy stays within
    1% with omega_p dt = 0.1, its error is the O(dt^2) error of the leapfrog
    (Sec. 1: the EC schemes conserve energy approximately at finite dt), while
    the momentum-conserving scheme heats steadily."""
    tot2, _ = _thermal_periodic("ec_explicit", 0.2, 5000)
    tot1, _ = _thermal_periodic("ec_explicit", 0.1, 10000)
    dev2 = np.max(np.abs(tot2 / tot2[0] - 1.0))
    dev1 = np.max(np.abs(tot1 / tot1[0] - 1.0))
    assert dev1 < 0.01
    assert 3.0 < dev2 / dev1 < 5.0
    _, ke_mc = _thermal_periodic("mc_explicit", 0.2, 5000)
    gain = ke_mc[-1] / ke_mc[0] - 1.0
    slope = np.polyfit(np.arange(len(ke_mc)), ke_mc / ke_mc[0], 1)[0]
    assert gain > 0.05 and slope > 0
    assert gain > 5 * dev2


def d1_roots(w):
    """Roots of (z-1)^2 (2z-1) + w^2 z^3 = 0, i.e. (2 + w^2) z^3 - 5 z^2 + 4 z - 1."""
    return np.roots([2.0 + w * w, -5.0, 4.0, -1.0])


@pytest.mark.parametrize("scheme", ["ec_implicit", "mc_implicit"])
@pytest.mark.parametrize("wdt", [0.5, 2.0, 5.0])
def test_direct_implicit_cold_oscillation_follows_d1_recurrence(wdt, scheme):
    n_cells, n0 = 128, 1e15
    dt = wdt / omega_p(n0)
    sim, _ = cold_plasma(n_cells, 16, n0, dt, 0.02, scheme=scheme)
    steps = 24 if wdt > 1 else 60
    a = np.real(run_series(sim, n_cells, steps))[1:]
    # Prony: fit a_{n+3} = c2 a_{n+2} + c1 a_{n+1} + c0 a_n, keep points above round-off
    keep = np.abs(a) > 1e-9 * np.abs(a).max()
    m = int(np.argmin(keep)) if not keep.all() else len(a)
    a = a[:m]
    A = np.stack([a[2:-1], a[1:-2], a[:-3]], axis=1)
    c = np.linalg.lstsq(A, a[3:], rcond=None)[0]
    fit = np.roots([1.0, -c[0], -c[1], -c[2]])
    theory = d1_roots(wdt)
    zt = theory[np.argmax(np.abs(theory))]
    zf = fit[np.argmax(np.abs(fit))]
    assert abs(zf) == pytest.approx(abs(zt), rel=5e-3)
    assert abs(np.angle(zf)) == pytest.approx(abs(np.angle(zt)), rel=5e-3, abs=1e-3)
    if wdt >= 5.0:
        assert abs(zt) < 0.75  # strong damping of the resolved oscillation
