"""Pins of the oracle's Monte Carlo collisions, random numbers, load and
electrode absorption (no GPU).  Sec. 3 describes the discharge model: uniform
initial plasma, electrodes that absorb, electron-atom and ion-atom collisions
(the method is the null-collision Monte Carlo of Vahedi & Surendra), no
secondary emission."""
import math

import numpy as np
import pytest
from scipy import stats

import oracle
import workloads

E = 1.602176634e-19
ME = 9.1093837015e-31
AMU = 1.66053906660e-27
KB = 1.380649e-23
TORR = 101325.0 / 760.0


def gas_density(mtorr, t=300.0):
    return mtorr * 1e-3 * TORR / (KB * t)


def speed(eps_ev, m=ME):
    return math.sqrt(2.0 * eps_ev * E / m)


def iso_dirs(rng, n):
    v = rng.standard_normal((n, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def box(**kw):
    """Periodic box without field (negligible macro weight), collisions on."""
    c = workloads.cfg_periodic(n_cells=16, np_e=1, n0=1e-6, length=0.016, dt=1e-10)
    c.update(dict(mcc=True, pressure_mtorr=30.0, gas_temp=300.0, quantized=False,
                  **workloads.CROSS_SECTIONS))
    c.update(kw)
    return c


def put(sim, species, v, rng, n_cells=16, ids=None):
    n = len(v)
    xi = rng.uniform(0, n_cells, n)
    ids = np.arange(n, dtype=np.uint32) if ids is None else ids
    sim.set_species(species, xi, v[:, 0], v[:, 1], v[:, 2], ids)
    return xi


# ---------------------------------------------------------------- Philox
def test_philox_output_statistics():
    w = oracle.philox_stream((1234, 5678), (0, 7, 0, 0), 250_000).ravel()
    counts = np.bincount((w >> 24).astype(np.int64), minlength=256)
    assert stats.chisquare(counts).pvalue > 1e-4
    bits = ((w[:, None] >> np.arange(32, dtype=np.uint32)) & 1).mean(axis=0)
    assert np.max(np.abs(bits - 0.5)) < 5 / math.sqrt(len(w))
    # successive words are uncorrelated
    u = w.astype(np.float64) / 2 ** 32
    assert abs(np.corrcoef(u[:-1], u[1:])[0, 1]) < 5 / math.sqrt(len(u))


def test_philox_avalanche_on_counter_and_key():
    rng = np.random.default_rng(0)
    flips = []
    for _ in range(200):
        key = rng.integers(0, 2 ** 32, 2, dtype=np.uint64).astype(np.uint32)
        ctr = rng.integers(0, 2 ** 32, 4, dtype=np.uint64).astype(np.uint32)
        base = oracle.philox(key, ctr)
        for word in range(4):
            c2 = ctr.copy()
            c2[word] ^= np.uint32(1 << int(rng.integers(0, 32)))
            diff = oracle.philox(key, c2) ^ base
            flips.append(sum(bin(int(x)).count("1") for x in diff))
        k2 = key.copy()
        k2[0] ^= np.uint32(1)
        diff = oracle.philox(k2, ctr) ^ base
        flips.append(sum(bin(int(x)).count("1") for x in diff))
    assert np.mean(flips) == pytest.approx(64.0, abs=1.5)


# ---------------------------------------------------------------- load
def test_uniform_maxwellian_load():
    """Sec. 3: the plasma starts uniform between the electrodes; velocities
    are Maxwellian at the load temperatures."""
    c = dict(workloads.CFG_SMALL_CCP, np_init=100_000, mcc=False)
    sim = oracle.Sim(c).load(100_000, 100_000)
    for sp, t_ev, m in (("e", c["te_ev"], ME), ("i", c["ti_ev"], c["ion_mass_amu"] * AMU)):
        s = sim.get_species(sp)
        assert np.array_equal(np.sort(s["id"]), np.arange(100_000))
        assert stats.kstest(s["xi"] / c["n_cells"], "uniform").pvalue > 1e-4
        vth = math.sqrt(E * t_ev / m)
        for comp in ("vx", "vy", "vz"):
            v = s[comp] / vth
            assert abs(v.mean()) < 5 / math.sqrt(len(v))
            assert v.var() == pytest.approx(1.0, rel=0.02)
            assert stats.kstest(v, "norm").pvalue > 1e-4
        # offsets carry 24 fractional bits: the device representation holds them exactly
        frac = s["xi"] * 2 ** 24
        assert np.array_equal(frac, np.round(frac))


def test_quasineutral_load_has_zero_net_charge_exactly():
    c = dict(workloads.CFG_SMALL_CCP, mcc=False)
    sim = oracle.Sim(c).load(12800, 12800)
    g = sim.grids()
    assert g["rho_q_e"].sum() == g["rho_q_i"].sum() == 12800 * 2 ** 33
    assert (g["rho_q_i"] - g["rho_q_e"]).sum() == 0


# ---------------------------------------------------------------- null collisions
def test_null_collision_waiting_time_is_geometric():
    """Constant cross section at fixed speed with the bound equal to the true
    rate: every selected particle collides, so the first collision step is
    geometric with p = 1 - exp(-n_g sigma v dt)."""
    eps_cap = 100.0
    n, dt, sig = 20_000, 2e-10, 1e-19
    c = box(sig_exc_max=0.0, sig_iz_peak=0.0, sig_el=sig, eps_cap=eps_cap, dt=dt,
            ion_mass_amu=1e9, np_init=n)
    sim = oracle.Sim(c, cap_e=n + 10, cap_i=10)
    rng = np.random.default_rng(1)
    v = iso_dirs(rng, n) * speed(eps_cap)
    put(sim, "e", v, rng)
    sim.set_species("i", [], [], [], [], np.zeros(0, dtype=np.uint32), next_id=0)
    sim.init_field()
    d = oracle.derive(c)
    p_theory = 1.0 - math.exp(-gas_density(30.0) * sig * speed(eps_cap) * dt)
    p = d["p_null_e"]
    assert abs(p - p_theory) <= 1e-12 * p_theory
    first = np.zeros(n, dtype=np.int64)
    prev = sim.get_species("e")
    order = np.argsort(prev["id"])
    prev_dir = np.stack([prev[k][order] for k in ("vx", "vy", "vz")], 1)
    steps = 80
    for k in range(1, steps + 1):
        sim.step(1)
        cur = sim.get_species("e")
        o = np.argsort(cur["id"])
        cd = np.stack([cur[q][o] for q in ("vx", "vy", "vz")], 1)
        changed = np.linalg.norm(cd - prev_dir, axis=1) > 1e-6 * speed(eps_cap)
        first[(first == 0) & changed] = k
        prev_dir = cd
    assert sim.diag()["coll"][4] == 0  # no null events: the bound equals the rate
    obs = np.bincount(first, minlength=steps + 1)
    exp_ = n * (1 - p) ** (np.arange(steps + 1) - 1) * p
    exp_[0] = n * (1 - p) ** steps
    assert stats.chisquare(obs, exp_).pvalue > 1e-4


WAIT_CAP = 64 ** 3
REDRAW = 1 << 30


def _wait_cfg(mtorr, dt):
    return box(pressure_mtorr=mtorr, dt=dt, np_init=1)


# P_null from 0.36 down to 5e-7 (where most draws reach the cap)
WAIT_CASES = [(30.0, 6e-10), (30.0, 1e-10), (30.0, 2e-12), (10.0, 1e-13), (0.3, 3e-13), (1.0, 2e-14)]


@pytest.mark.parametrize("mtorr,dt", WAIT_CASES)
def test_waiting_time_tables_compose_to_the_geometric_law(mtorr, dt):
    """Selection by waiting times: W - 1 = X = 4096 a + 64 b + c from three
    independent digits, each the number of thresholds above a 32-bit word.
    From the tables alone, P(X >= x) = P(a > a') + P(a = a') (P(b > b') +
    P(b = b') P(c >= c')) must equal q^x, q = 1 - P_null, for every x below the
    cap (here a spread of x from one step to past 64^3), and P(a = 64) must be
    q^(64^3): a wrong ratio, an off-by-one threshold or a wrong digit weight
    breaks this identity.  Exact up to the 2^-32 rounding of each threshold."""
    c = _wait_cfg(mtorr, dt)
    d = oracle.derive(c)
    P = d["p_null_e"]
    assert 1e-7 < P < 0.4
    q = 1.0 - P
    t = d["wait_thr"][0].astype(np.float64) / 2 ** 32  # [digit c, b, a][j - 1]

    def ge(digit, j, n):  # P(digit >= j), j in 0..n
        return 1.0 if j == 0 else (0.0 if j > n else t[digit][j - 1])

    xs = sorted({0, 1, 2, 3, 31, 63, 64, 65, 127, 4095, 4096, 4097, 12345, 99999, 262143}
                | set(range(0, 400, 7)))
    for x in xs:
        a, b, cc = x // 4096, (x // 64) % 64, x % 64
        pa_gt = ge(2, a + 1, 64)
        pa_eq = ge(2, a, 64) - ge(2, a + 1, 64)
        pb_gt = ge(1, b + 1, 63)
        pb_eq = ge(1, b, 63) - ge(1, b + 1, 63)
        pc_ge = ge(0, cc, 63)
        got = pa_gt + pa_eq * (pb_gt + pb_eq * pc_ge)
        assert abs(got - q ** x) <= 6 * 2 ** -32, (x, got, q ** x)
    assert abs(ge(2, 64, 64) - q ** WAIT_CAP) <= 2 * 2 ** -32


@pytest.mark.parametrize("mtorr,dt", [(30.0, 1e-10), (10.0, 1e-13), (0.3, 3e-13)])
def test_waiting_time_draws_follow_the_geometric_law(mtorr, dt):
    """Drawn waits (entry draws of 300,000 ids) against the geometric law
    P(W = k) = q^(k-1) P_null: chi-square over bins of equal probability, and
    the share of capped draws (a count of 64^3 steps marked for a fresh draw)
    equal to q^(64^3)."""
    c = _wait_cfg(mtorr, dt)
    P = oracle.derive(c)["p_null_e"]
    q = 1.0 - P
    n = 300_000
    w = oracle.wait_draws(c, "e", np.arange(n, dtype=np.uint32), step=17, sub=1).astype(np.int64)
    capped = (w & REDRAW) != 0
    assert np.all((w[capped] & ~REDRAW) == WAIT_CAP)
    p_cap = q ** WAIT_CAP
    assert abs(capped.mean() - p_cap) <= 5 * math.sqrt(p_cap * (1 - p_cap) / n) + 1e-12
    W = w[~capped]
    assert W.min() >= 1 and W.max() <= WAIT_CAP
    # 20 bins of equal probability under the law cut at the cap
    edges = [1]
    for j in range(1, 20):  # P(W > k) = q^k: the k that leaves 1 - j/20 of the uncut part above it
        k = math.log(1 - (1 - p_cap) * j / 20) / math.log(q)
        edges.append(int(math.floor(k)) + 1)
    edges.append(WAIT_CAP + 1)
    edges = sorted(set(edges))
    obs = np.histogram(W, bins=edges)[0]
    cdf = lambda k: 1.0 - q ** (k - 1)  # P(W < k)
    exp_ = np.array([cdf(edges[i + 1]) - cdf(edges[i]) for i in range(len(edges) - 1)]) * n
    exp_ *= obs.sum() / exp_.sum()
    assert stats.chisquare(obs, exp_).pvalue > 1e-4
    assert abs(W.mean() - (1 / P)) < 6 * math.sqrt(q) / P / math.sqrt(len(W)) + (1 / P) * p_cap * 2


def test_waiting_time_draws_are_keyed_on_id_step_and_kind():
    """Draws depend on (id, step, entry or reselection) and nothing else:
    repeated calls agree, and changing any key gives a different stream."""
    c = _wait_cfg(30.0, 1e-10)
    ids = np.arange(5000, dtype=np.uint32)
    a = oracle.wait_draws(c, "e", ids, step=3, sub=1)
    assert np.array_equal(a, oracle.wait_draws(c, "e", ids, step=3, sub=1))
    for other in (oracle.wait_draws(c, "e", ids, step=4, sub=1), oracle.wait_draws(c, "e", ids, step=3, sub=0),
                  oracle.wait_draws(c, "i", ids, step=3, sub=1), oracle.wait_draws(c, "e", ids + 1, step=3, sub=1)):
        assert np.mean(a != other) > 0.9


def test_process_frequencies_follow_cross_sections():
    """Electrons at eps = e * I, where the ionisation cross section takes its
    stated peak 3e-20 m^2 and excitation sits on its plateau, with the bound
    taken at the same energy (the bound is then n_g v (sigma_el + sigma_exc,max
    + sigma_iz,peak)): selected electrons choose elastic / excitation /
    ionisation in proportion to their cross sections, and no null event."""
    cs = workloads.CROSS_SECTIONS
    eps = math.e * cs["iz_thr"]
    n = 400_000
    c = box(eps_cap=eps, dt=1e-10, np_init=n)
    sim = oracle.Sim(c, cap_e=2 * n, cap_i=2 * n)
    rng = np.random.default_rng(2)
    put(sim, "e", iso_dirs(rng, n) * speed(eps), rng)
    sim.set_species("i", [], [], [], [], np.zeros(0, dtype=np.uint32), next_id=0)
    sim.init_field()
    ng = gas_density(30.0)
    sig = np.array([cs["sig_el"], cs["sig_exc_max"], cs["sig_iz_peak"]])
    nu_max = ng * speed(eps) * sig.sum()
    d = oracle.derive(c)
    assert d["nu_max_e"] == pytest.approx(nu_max, rel=1e-12)
    assert d["p_null_e"] == pytest.approx(1 - math.exp(-nu_max * 1e-10), rel=1e-12)
    sim.step(1)
    coll = sim.diag()["coll"]
    ps = d["thr_e"] / 2 ** 24
    probs = np.array([1 - ps, *(ps * sig / sig.sum())])
    obs = np.array([n - sum(coll[:3]) - coll[4], coll[0], coll[1], coll[2]])
    assert coll[4] == 0
    assert stats.chisquare(obs, probs * n).pvalue > 1e-4
    assert sim.count("e") == n + coll[2] and sim.count("i") == coll[2]


def test_collision_bound_covers_every_energy_below_cap():
    """The null-collision bound must not be exceeded below eps_cap: the
    selected-and-real fraction never saturates (no overflow counted) for
    electrons spread over (0, eps_cap)."""
    n = 200_000
    c = box(np_init=n, dt=1e-10)
    sim = oracle.Sim(c, cap_e=2 * n, cap_i=2 * n)
    rng = np.random.default_rng(12)
    eps = rng.uniform(0.01, 100.0, n)
    put(sim, "e", iso_dirs(rng, n) * np.sqrt(2 * eps * E / ME)[:, None], rng)
    sim.set_species("i", [], [], [], [], np.zeros(0, dtype=np.uint32), next_id=0)
    sim.init_field()
    sim.step(1)
    d = sim.diag()
    assert d["overflow"][0] == 0 and d["coll"][4] > 0


def test_rotation_geometry_and_isotropy():
    rng = np.random.default_rng(3)
    dirs = list(iso_dirs(rng, 20)) + [np.array([1.0, 0, 0]), np.array([-1.0, 0, 0]),
                                      np.array([1.0, 1e-8, 0]) / math.hypot(1, 1e-8)]
    for d in dirs:
        for _ in range(20):
            cc = rng.uniform(-1, 1)
            ph = rng.uniform(0, 2 * math.pi)
            out = oracle.rotate(d, cc, ph)
            assert np.linalg.norm(out) == pytest.approx(1.0, abs=1e-12)
            # within 1e-6 of the x axis the limiting basis is used: error O(sin theta)
            tol = 1e-9 if math.hypot(d[1], d[2]) > 1e-6 else 2e-6
            assert float(out @ d) == pytest.approx(cc, abs=tol)
    # uniform cos(chi) and azimuth give isotropic directions for any incident d
    for d in (dirs[0], np.array([1.0, 0, 0])):
        outs = np.array([oracle.rotate(d, rng.uniform(-1, 1), rng.uniform(0, 2 * math.pi))
                         for _ in range(20000)])
        assert np.max(np.abs(outs.mean(0))) < 0.03
        np.testing.assert_allclose(outs.T @ outs / len(outs), np.eye(3) / 3, atol=0.02)


def _one_step_beam(eps, n, seed, **kw):
    c = box(np_init=n, **kw)
    sim = oracle.Sim(c, cap_e=2 * n, cap_i=2 * n)
    rng = np.random.default_rng(seed)
    v = iso_dirs(rng, n) * speed(eps)
    xi = put(sim, "e", v, rng)
    sim.set_species("i", [], [], [], [], np.zeros(0, dtype=np.uint32), next_id=0)
    sim.init_field()
    sim.step(1)
    return sim, c, v, xi


def test_elastic_energy_loss_and_isotropy():
    """Elastic scattering is isotropic and the electron keeps the fraction
    1 - (2m/M)(1 - cos chi) of its energy (mean loss 2m/M)."""
    M = 0.01 * AMU
    sim, c, v0, _ = _one_step_beam(10.0, 100_000, 4, sig_exc_max=0.0, sig_iz_peak=0.0,
                                   ion_mass_amu=0.01, dt=2e-9)
    s = sim.get_species("e")
    o = np.argsort(s["id"])
    v1 = np.stack([s[k][o] for k in ("vx", "vy", "vz")], 1)
    moved = np.linalg.norm(v1 - v0, axis=1) > 1e-6 * speed(10.0)
    assert moved.sum() == sim.diag()["coll"][0] > 5000
    a, b = v0[moved], v1[moved]
    cos_chi = np.sum(a * b, 1) / (np.linalg.norm(a, axis=1) * np.linalg.norm(b, axis=1))
    ratio = np.sum(b * b, 1) / np.sum(a * a, 1)
    np.testing.assert_allclose(ratio, 1 - 2 * ME / M * (1 - cos_chi), rtol=1e-9)
    assert abs(cos_chi.mean()) < 5 / math.sqrt(len(cos_chi))
    assert np.mean(cos_chi ** 2) == pytest.approx(1 / 3, abs=5 * 0.3 / math.sqrt(len(cos_chi)))
    assert ratio.mean() == pytest.approx(1 - 2 * ME / M, abs=5 * 0.07 / math.sqrt(len(ratio)))


def test_excitation_removes_threshold_energy():
    cs = workloads.CROSS_SECTIONS
    sim, c, v0, _ = _one_step_beam(30.0, 50_000, 5, sig_el=0.0, sig_iz_peak=0.0, dt=2e-9)
    s = sim.get_species("e")
    o = np.argsort(s["id"])
    v1 = np.stack([s[k][o] for k in ("vx", "vy", "vz")], 1)
    e1 = 0.5 * ME * np.sum(v1 * v1, 1) / E
    hit = np.abs(e1 - 30.0) > 1e-6
    assert hit.sum() == sim.diag()["coll"][1] > 1000
    np.testing.assert_allclose(e1[hit], 30.0 - cs["exc_thr"], rtol=1e-9)


def test_ionisation_creates_one_pair_shares_energy_and_ranks_child_ids():
    """Ionisation removes the threshold, the two electrons share what is left
    equally (reading), a new ion appears at the parent's position, and the
    children of the step get consecutive ids in increasing parent id."""
    cs = workloads.CROSS_SECTIONS
    n = 50_000
    sim, c, v0, xi0 = _one_step_beam(60.0, n, 6, sig_el=0.0, sig_exc_max=0.0, dt=2e-9)
    nb = sim.diag()["coll"][2]
    assert nb > 1000 and sim.count("e") == n + nb and sim.count("i") == nb
    e = sim.get_species("e")
    ions = sim.get_species("i")
    share = 0.5 * (60.0 - cs["iz_thr"])
    parent = e["id"] < n
    en = 0.5 * ME * (e["vx"] ** 2 + e["vy"] ** 2 + e["vz"] ** 2) / E
    changed = parent & (np.abs(en - 60.0) > 1e-6)
    assert changed.sum() == nb
    np.testing.assert_allclose(en[changed], share, rtol=1e-9)
    np.testing.assert_allclose(en[~parent], share, rtol=1e-9)
    # children sit at their parent's position; ids ranked by parent id
    pid_sorted = np.sort(e["id"][changed])
    pos_of_parent = dict(zip(e["id"][changed].tolist(), e["xi"][changed].tolist()))
    child_pos = dict(zip(e["id"][~parent].tolist(), e["xi"][~parent].tolist()))
    ion_pos = dict(zip(ions["id"].tolist(), ions["xi"].tolist()))
    for rank, pid in enumerate(pid_sorted.tolist()):
        assert child_pos[n + rank] == pos_of_parent[pid]
        assert ion_pos[rank] == pos_of_parent[pid]


def test_charge_exchange_gives_gas_maxwellian():
    n = 200_000
    c = box(np_init=n, ions_mobile=True, dt=5e-8, cx_vmax=200.0)
    sim = oracle.Sim(c, cap_e=16, cap_i=n + 16)
    rng = np.random.default_rng(7)
    v = np.tile([2.0e4, 0.0, 0.0], (n, 1))
    sim.set_species("e", [], [], [], [], np.zeros(0, dtype=np.uint32), next_id=0)
    put(sim, "i", v, rng)
    sim.init_field()
    sim.step(1)
    s = sim.get_species("i")
    hit = np.abs(s["vx"] - 2.0e4) > 1e-6
    assert hit.sum() == sim.diag()["coll"][3] > 5000
    vth = math.sqrt(KB * 300.0 / (39.948 * AMU))
    # The null-collision method accepts a sampled neutral with probability
    # proportional to the relative speed g, so the ion leaves with the
    # g-weighted gas Maxwellian: its moments from a large independent sample.
    ref = np.random.default_rng(70).standard_normal((4_000_000, 3)) * vth
    g = np.linalg.norm(ref - v[0], axis=1)
    for k, comp in enumerate(("vx", "vy", "vz")):
        u = s[comp][hit]
        m_ref = np.sum(g * ref[:, k]) / g.sum()
        v_ref = np.sum(g * (ref[:, k] - m_ref) ** 2) / g.sum()
        assert abs(u.mean() - m_ref) < 5 * vth / math.sqrt(len(u))
        assert u.var() == pytest.approx(v_ref, rel=5 * math.sqrt(2.0 / len(u)))
    assert np.sum(g * ref[:, 0]) / g.sum() < -0.5 * vth ** 2 / 2.0e4  # the bias is real


# ---------------------------------------------------------------- electrodes
def test_electrode_absorption_counts_and_energy():
    """Sec. 3: particles that reach an electrode are absorbed (no secondary
    emission); the wall tally gets their number and kinetic energy."""
    n_cells, L, dt = 32, 0.032, 1e-9
    c = dict(workloads.CFG_SMALL_CCP, n_cells=n_cells, length=L, dt=dt, mcc=False, n0=1e-6,
             np_init=1000, rf_volt=0.0, quantized=False)
    sim = oracle.Sim(c, cap_e=2000, cap_i=2000)
    rng = np.random.default_rng(8)
    n = 1000
    xi = rng.uniform(0, 3, n)
    vx = -rng.uniform(0, 3e6, n)
    vy = rng.normal(0, 1e5, n)
    vz = rng.normal(0, 1e5, n)
    sim.set_species("e", xi, vx, vy, vz, np.arange(n, dtype=np.uint32))
    xi_i = rng.uniform(n_cells - 2, n_cells, n)
    vi = rng.uniform(0, 5e4, n)
    sim.set_species("i", xi_i, vi, vy, vz, np.arange(n, dtype=np.uint32))
    sim.init_field()
    sim.step(1)
    dx = L / n_cells
    gone_e = xi + vx * dt / dx < 0
    gone_i = xi_i + vi * dt / dx >= n_cells
    d = sim.diag()
    assert d["wall_count"][0] == [int(gone_e.sum()), 0]
    assert d["wall_count"][1] == [0, int(gone_i.sum())]
    en = 0.5 * ME * (vx ** 2 + vy ** 2 + vz ** 2) / E
    assert d["wall_energy_ev"][0][0] == pytest.approx(en[gone_e].sum(), rel=1e-9)
    assert sim.count("e") == n - gone_e.sum() and sim.count("i") == n - gone_i.sum()


def test_eedf_counts_every_electron_in_its_bin():
    c = box(np_init=5000, mcc=False, diag_period=1, eedf_bins=50, eedf_max_ev=50.0)
    sim = oracle.Sim(c, cap_e=6000, cap_i=16)
    rng = np.random.default_rng(9)
    eps = rng.uniform(0.2, 60.0, 5000)
    eps[np.abs(eps - np.round(eps)) < 1e-3] += 0.01
    v = iso_dirs(rng, 5000) * np.sqrt(2 * eps * E / ME)[:, None]
    put(sim, "e", v, rng)
    sim.set_species("i", [], [], [], [], np.zeros(0, dtype=np.uint32), next_id=0)
    sim.init_field()
    sim.step(1)
    h = sim.averages()["eedf"]
    assert h.sum() == 5000
    ref = np.bincount(np.minimum(np.floor(eps).astype(int), 50), minlength=51)
    assert np.array_equal(h, ref)


# ---------------------------------------------------------------- collision model options
def _vs_law(eps):
    """The Vahedi-Surendra law as a density in mu = cos chi: the screened
    Coulomb differential cross section ~ 1 / (1 + eps sin^2(chi/2)) per solid
    angle, sin^2(chi/2) = (1 - mu)/2; normalised by quadrature."""
    from scipy import integrate
    f = lambda mu: 1.0 / (1.0 + eps * (1.0 - mu) / 2.0)
    z = integrate.quad(f, -1.0, 1.0)[0]
    mom = lambda k: integrate.quad(lambda mu: mu ** k * f(mu), -1.0, 1.0)[0] / z
    cdf = np.vectorize(lambda m: integrate.quad(f, -1.0, m)[0] / z)
    return mom(1), mom(2), cdf


@pytest.mark.parametrize("eps", [0.5, 5.0, 30.0, 120.0])
def test_vahedi_surendra_angles_follow_their_cross_section(eps):
    """Sampled cos chi against the law integrated from its differential cross
    section (an independent route from the inverse-CDF formula): first and
    second moments within 5 sigma, and a Kolmogorov-Smirnov test."""
    u = np.random.default_rng(int(eps * 10)).uniform(0.0, 1.0, 40_000)
    mu = oracle.vs_cos_chi(eps, u)
    assert np.all(mu >= -1.0 - 1e-12) and np.all(mu <= 1.0 + 1e-12)
    m1, m2, cdf = _vs_law(eps)
    se = np.std(mu) / math.sqrt(len(mu))
    assert abs(mu.mean() - m1) < 5 * se, (mu.mean(), m1)
    assert abs((mu ** 2).mean() - m2) < 5 * np.std(mu ** 2) / math.sqrt(len(mu))
    assert stats.kstest(mu[:4000], cdf).pvalue > 1e-4
    # low energy tends to isotropy, high energy to forward scattering
    assert (m1 > 0.3) == (eps > 5.0)


@pytest.mark.parametrize("excess,b", [(5.0, 10.0), (44.2, 10.0), (200.0, 10.0)])
def test_opal_secondary_energy_law(excess, b):
    """Secondary energies of the Opal-Pollock-Wagner spectrum ~ 1/(1 + (e/B)^2)
    on [0, excess/2]: the mean B ln(1 + x^2) / (2 arctan x), x = excess/(2B)
    (closed form), and a Kolmogorov-Smirnov test against the CDF
    arctan(e/B) / arctan(x)."""
    u = np.random.default_rng(3).uniform(0.0, 1.0, 60_000)
    es = oracle.opal_secondary(excess, b, u)
    assert es.min() >= 0.0 and es.max() <= excess / 2 + 1e-12
    x = excess / (2 * b)
    mean = b * math.log(1 + x * x) / (2 * math.atan(x))
    assert abs(es.mean() - mean) < 5 * es.std() / math.sqrt(len(es))
    assert stats.kstest(es[:5000], lambda e: np.arctan(e / b) / math.atan(x)).pvalue > 1e-4


def test_opal_split_conserves_the_excess_in_a_run():
    """With the Opal split the primary and its secondary leave an ionisation
    with energies that add up to eps - I, the secondary below (eps - I)/2."""
    cs = workloads.CROSS_SECTIONS
    n = 50_000
    sim, c, v0, xi0 = _one_step_beam(60.0, n, 6, sig_el=0.0, sig_exc_max=0.0, dt=2e-9, iz_split="opal",
                                     iz_split_b=10.0)
    nb = sim.diag()["coll"][2]
    assert nb > 1000 and sim.count("e") == n + nb
    e = sim.get_species("e")
    en = 0.5 * ME * (e["vx"] ** 2 + e["vy"] ** 2 + e["vz"] ** 2) / E
    parent = e["id"] < n
    changed = parent & (np.abs(en - 60.0) > 1e-6)
    assert changed.sum() == nb
    pid_sorted = np.sort(e["id"][changed])
    e_par = dict(zip(e["id"][changed].tolist(), en[changed].tolist()))
    e_chi = dict(zip(e["id"][~parent].tolist(), en[~parent].tolist()))
    excess = 60.0 - cs["iz_thr"]
    for rank, pid in enumerate(pid_sorted.tolist()):
        assert abs(e_par[pid] + e_chi[n + rank] - excess) < 1e-9 * excess
        assert e_chi[n + rank] <= excess / 2 + 1e-9
    x = excess / 20.0
    mean = 10.0 * math.log(1 + x * x) / (2 * math.atan(x))
    sec = np.array(list(e_chi.values()))
    assert abs(sec.mean() - mean) < 5 * sec.std() / math.sqrt(len(sec))


def test_vahedi_surendra_elastic_deflection_in_a_run():
    """Elastic scattering with the anisotropic law: the mean cosine between
    incident and scattered directions of 30 eV electrons equals the law's mean
    at 30 eV, and the energy kept is 1 - (2m/M)(1 - cos chi) per electron."""
    sim, c, v0, _ = _one_step_beam(30.0, 100_000, 8, sig_exc_max=0.0, sig_iz_peak=0.0, ion_mass_amu=0.01,
                                   dt=2e-9, scattering="vahedi_surendra")
    s = sim.get_species("e")
    o = np.argsort(s["id"])
    v1 = np.stack([s[k][o] for k in ("vx", "vy", "vz")], 1)
    moved = np.linalg.norm(v1 - v0, axis=1) > 1e-6 * speed(30.0)
    assert moved.sum() == sim.diag()["coll"][0] > 5000
    a, b = v0[moved], v1[moved]
    cos_chi = np.sum(a * b, 1) / (np.linalg.norm(a, axis=1) * np.linalg.norm(b, axis=1))
    m1, _, _ = _vs_law(30.0)
    assert abs(cos_chi.mean() - m1) < 5 * cos_chi.std() / math.sqrt(len(cos_chi))
    ratio = np.sum(b * b, 1) / np.sum(a * a, 1)
    two_m_over_M = 2 * ME / (0.01 * AMU)
    np.testing.assert_allclose(ratio, 1 - two_m_over_M * (1 - cos_chi), rtol=0, atol=1e-9)
