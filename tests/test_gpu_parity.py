"""GPU path (libpic.so through its C ABI) against the CPU oracle, element by
element on the same seeded inputs.

Bars (written in each test):
* integer work bit-exact: Philox words, the uniform load's cells and
  offsets, the int64 node charge of an injected state, particle counts,
  collision / birth / wall tallies on the same Philox stream;
* floating point within the stated tolerance: positions |dx| <= 1e-5 L and
  velocities |dv| <= 1e-5 max(|v|, v_th) per particle after up to 100 steps
  (FP32 push against the FP64 oracle), fields within 1e-9 of their scale.
"""
import math

import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu

E = 1.602176634e-19
ME = 9.1093837015e-31
AMU = 1.66053906660e-27
NODE_DECISIONS = 4  # particles per species a non-uniform grid's node decisions may set apart (see compare_particles)


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def with_grid(cfg):
    """A configuration with `grid_beta` gets the stretched grid of that beta
    (non-uniform cells, Sec. 4) as its cell widths."""
    if cfg.get("grid_beta") is not None and cfg.get("cell_width") is None:
        cfg = dict(cfg, cell_width=workloads.stretched_widths(cfg["n_cells"], cfg["length"], cfg["grid_beta"]))
    return cfg


def node_lengths(cfg, dx):
    """The length a node's charge is spread over in the densities: dx, or on
    a non-uniform grid (h_{g-1} + h_g)/2 (wall nodes: their one cell;
    periodic: wrapped)."""
    if cfg.get("cell_width") is None:
        return dx
    h = np.asarray(cfg["cell_width"], dtype=np.float64)
    n = h.size
    g = np.arange(n + 1)
    if cfg.get("periodic"):
        return 0.5 * (h[(g - 1) % n] + h[g % n])
    return 0.5 * (h[np.maximum(g - 1, 0)] + h[np.minimum(g, n - 1)])


def gpu_sim(cfg):
    from paper_1310_5284_gb300.sim import Sim
    return Sim(cfg, device="cuda:0")


def vth(cfg, k):
    m = ME if k == 0 else cfg.get("ion_mass_amu", 39.948) * AMU
    t = cfg.get("te_ev", 2.0) if k == 0 else cfg.get("ti_ev", 0.026)
    return math.sqrt(E * t / m)


def inject(gpu, orc, cfg, states, step=0, abar=None):
    """Same seeded state into both: the GPU gets the storage form, the oracle
    the exact FP64 values of it (position in cell units = cell + offset)."""
    for k, sp in enumerate(("e", "i")):
        s = states[k]
        if s is None:
            continue
        ab = None if abar is None else abar[k]
        gpu.set_particles(sp, dict(s, abar=ab), next_id=int(s["id"].max()) + 1 if len(s["id"]) else 0)
        orc.set_species(sp, workloads.xi_of(s), s["vx"].astype(np.float64), s["vy"].astype(np.float64),
                        s["vz"].astype(np.float64), s["id"], abar=None if ab is None else ab.astype(np.float64),
                        next_id=int(s["id"].max()) + 1 if len(s["id"]) else 0)
    gpu.set_step(step)
    orc.set_step(step)
    gpu.init_field(set_abar=abar is None)
    orc.init_field(set_abar=abar is None)


def states_for(cfg, n, seed, sorted_cells=False, ions=True):
    st_e = workloads.injected_particles(seed, n, cfg["n_cells"], vth(cfg, 0), sorted_cells=sorted_cells)
    st_i = workloads.injected_particles(seed + 1, n, cfg["n_cells"], vth(cfg, 1), sorted_cells=sorted_cells) if ions else None
    return [st_e, st_i]


def by_id(d, xi_key=None):
    o = np.argsort(d["id"])
    return {k: (v[o] if isinstance(v, np.ndarray) else v) for k, v in d.items()}


def _divergence(a, b, cfg, k):
    """Per-particle |dx| (cells) and |dv| / max(|v|, v_th) of two id-sorted states."""
    xa = a["cell"].astype(np.float64) + a["off"].astype(np.float64) if "cell" in a else a["xi"]
    dxi = np.abs(xa - b["xi"])
    if cfg.get("periodic"):
        dxi = np.minimum(dxi, cfg["n_cells"] - dxi)
    dv = np.zeros_like(dxi)
    for comp in ("vx", "vy", "vz"):
        bound = np.maximum(np.abs(b[comp]), vth(cfg, k))
        dv = np.maximum(dv, np.abs(a[comp].astype(np.float64) - b[comp]) / bound)
    return dxi, dv


def compare_particles(gpu, orc, cfg, tol=1e-5, species=("e", "i"), quantile=1.0, max_tol=None, floor=None):
    """Per particle |dx| <= tol L and |dv| <= tol max(|v|, v_th), for every
    particle (quantile 1) or the given quantile with all within max_tol.
    With `floor` (the oracle's own FP32 sensitivity, see fp32_sensitivity)
    the 99th percentile and the maximum may reach the floor instead."""
    for k, sp in enumerate(species):
        a = by_id(gpu.get_particles(sp))
        b = by_id(orc.get_species(sp))
        assert np.array_equal(a["id"], b["id"]), "particle sets differ (%s)" % sp
        if len(a["id"]) == 0:
            continue
        dxi, dv = _divergence(a, b, cfg, k)
        lim_x = tol * cfg["n_cells"]
        if floor is not None:
            f = floor[k]
            assert np.quantile(dxi, 0.99) <= max(lim_x, f["x99"]), ("x q99", sp, np.quantile(dxi, 0.99), f)
            assert np.quantile(dv, 0.99) <= max(tol, f["v99"]), ("v q99", sp, np.quantile(dv, 0.99), f)
            # On a non-uniform grid the force jumps at a node by the ratio of
            # the two widths, so which side of a node FP32 and FP64 put a
            # particle is a decision like a threshold's: the maxima hold for
            # all but the few particles furthest apart (NODE_DECISIONS).
            skip = NODE_DECISIONS if cfg.get("cell_width") is not None else 0
            xmax = np.sort(dxi)[-1 - skip] if len(dxi) > skip else 0.0
            vmax = np.sort(dv)[-1 - skip] if len(dv) > skip else 0.0
            assert xmax <= max(lim_x, f["xmax"]), ("x max", sp, xmax, f)
            assert vmax <= max(tol, f["vmax"]), ("v max", sp, vmax, f)
            continue
        assert np.quantile(dxi, quantile) <= lim_x, ("x", sp, float(np.quantile(dxi, quantile)))
        assert np.quantile(dv, quantile) <= tol, ("v", sp, float(np.quantile(dv, quantile)))
        if max_tol is not None:
            assert dxi.max() <= max_tol * cfg["n_cells"] and dv.max() <= max_tol, ("max", sp, dxi.max(), dv.max())


def fp32_sensitivity(cfg, states, steps, abar=None, factor=4.0, step0=0, next_ids=None, ulps=2):
    """The oracle's FP32 sensitivity (fp32_sensitivity_once); on a
    non-uniform grid the largest over two rounding realisations, since the
    force jumps at the nodes make one realisation's divergence vary by up to
    ten times from another's in chaotic cases."""
    seeds = (12345, 777) if cfg.get("cell_width") is not None else (12345,)
    runs = [fp32_sensitivity_once(cfg, states, steps, abar, factor, step0, next_ids, ulps, seed) for seed in seeds]
    out = []
    for k in range(len(runs[0])):
        fs = [r[k] for r in runs]
        if any(f is None for f in fs):
            out.append(None)
            continue
        out.append({key: (all(f[key] for f in fs) if key == "same_set" else max(f[key] for f in fs))
                    for key in fs[0]})
    return out


def fp32_sensitivity_once(cfg, states, steps, abar=None, factor=4.0, step0=0, next_ids=None, ulps=2, seed=12345):
    """How far the FP64 oracle drifts from itself when its particle state is
    put through the FP32 arithmetic of a device step after every step: the
    state is rounded to the storage form (cell + FP32 offset, FP32
    velocities) and each stored value moved by a seeded random whole number
    of FP32 ulps in [-ulps, ulps], the size of the few roundings the push
    makes per value (acceleration, velocity, displacement, renormalisation;
    in the implicit push, predictor and corrector).  This is the chaotic
    amplification of FP32 arithmetic alone, over the same Philox streams as
    the test (same first step and next ids), compared over the ids both runs
    hold.  Returns per species the floor (factor times the 99th percentile
    and the maximum of |dx| in cells and of |dv| / max(|v|, v_th)), plus the
    relative change that this makes to the kinetic energy of each species."""
    ref = oracle.Sim(cfg)
    rnd = oracle.Sim(cfg)
    nid = list(next_ids) if next_ids is not None else [None, None]
    for s in (ref, rnd):
        for k, sp in enumerate(("e", "i")):
            st = states[k]
            if st is None:
                continue
            if nid[k] is None:
                nid[k] = int(st["id"].max()) + 1 if len(st["id"]) else 0
            ab = None if abar is None or abar[k] is None else abar[k].astype(np.float64)
            s.set_species(sp, workloads.xi_of(st), st["vx"].astype(np.float64), st["vy"].astype(np.float64),
                          st["vz"].astype(np.float64), st["id"], abar=ab, next_id=nid[k])
        s.set_step(step0)
        s.init_field(set_abar=abar is None)
    births0 = rnd.diag()["births"]
    ref.step(steps)
    rng = np.random.default_rng(seed)

    def f32(x):
        y = np.asarray(x, dtype=np.float32)
        if ulps:
            y = y + np.spacing(y) * rng.integers(-ulps, ulps + 1, y.shape).astype(np.float32)
        return y.astype(np.float64)

    for _ in range(steps):
        rnd.step(1)
        born = rnd.diag()["births"] - births0
        for k, sp in enumerate(("e", "i")):
            d = rnd.get_species(sp)
            if len(d["id"]) == 0:
                continue
            c = np.floor(d["xi"])
            o = np.clip(f32(d["xi"] - c), 0.0, np.nextafter(np.float32(1.0), np.float32(0.0)))
            rnd.set_species(sp, c + o, f32(d["vx"]), f32(d["vy"]), f32(d["vz"]), d["id"], abar=f32(d["abar"]),
                            next_id=int(nid[k] + born), wait=d["wait"])
        rnd.init_field(set_abar=False)
    out = []
    da, db = rnd.diag(), ref.diag()
    for k, sp in enumerate(("e", "i")):
        a, b = by_id(rnd.get_species(sp)), by_id(ref.get_species(sp))
        common, ia, ib = np.intersect1d(a["id"], b["id"], assume_unique=True, return_indices=True)
        if len(common) == 0:
            out.append(None)
            continue
        a = {key: v[ia] for key, v in a.items()}
        b = {key: v[ib] for key, v in b.items()}
        dxi, dv = _divergence(a, b, cfg, k)
        ke = abs(da["ke_x"][k] - db["ke_x"][k]) / max(abs(db["ke_x"][k]), 1e-300)
        ab = np.abs(a["abar"] - b["abar"]).max() / max(np.abs(b["abar"]).max(), 1e-300)
        out.append(dict(x99=factor * np.quantile(dxi, 0.99), v99=factor * np.quantile(dv, 0.99),
                        xmax=factor * dxi.max(), vmax=factor * dv.max(), ke=ke, abar=factor * ab,
                        same_set=len(common) == len(rnd.get_species(sp)["id"]) == len(ref.get_species(sp)["id"])))
    return out


def ke_bar(tol, floor):
    """Relative bar on the kinetic energy of a species implied by the
    per-particle one: with |dv| <= t max(|v|, v_th) for every particle,
    |d(v^2)| <= 2 t (v^2 + v_th |v|), and the sum over particles stays within
    2 t (1 + <v_th |v|> / <v^2>) <= 4 t of the total (|v| is of order v_th
    on average)."""
    t = tol if floor is None else max(tol, floor["vmax"])
    return 4.0 * t


def _oracle_of(cfg, st, step, implicit, extra=4096):
    """An oracle run holding the given device-form state at the given step,
    with the field of that state."""
    orc = oracle.Sim(cfg, cap_e=len(st[0]["id"]) + extra, cap_i=len(st[1]["id"]) + extra)
    orc.set_step(step)  # particles entering at `step` draw their waits there, as uploads to the GPU do
    for k, sp in enumerate(("e", "i")):
        x = st[k]
        orc.set_species(sp, workloads.xi_of(x), x["vx"].astype(np.float64), x["vy"].astype(np.float64),
                        x["vz"].astype(np.float64), x["id"],
                        abar=x["abar"].astype(np.float64) if implicit else None, next_id=x["next_id"])
    orc.init_field(set_abar=False)
    return orc


def _rel(a, b):
    """Largest relative difference of a against b (elementwise)."""
    a, b = np.atleast_1d(np.asarray(a, dtype=np.float64)), np.atleast_1d(np.asarray(b, dtype=np.float64))
    return float((np.abs(a - b) / np.maximum(np.abs(b), 1e-300)).max()) if a.size else 0.0


def _of_scale(a, b):
    """Largest difference of a against b relative to max |b|."""
    a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)) if a.size else 0.0


def one_step_diagnostics(gpu, cfg, eedf_tol=None):
    """Every diagnostic of the GPU's next step against one oracle step taken
    from the GPU's own state (FP32 storage read exactly into FP64), so the
    plasma's chaos plays no part and the bars follow from FP32 arithmetic:
    * counts, wall counts, collision and birth tallies exact (integer
      decisions on the same Philox words);
    * kinetic energy, wall energy and the energy of the field the push used
      within 1e-5 relative (FP32 velocities carry 6e-8 of rounding, and FP32
      sums of a few hundred terms per thread a few 1e-7 more);
    * power and the J.E heating profile within 1e-5 of their magnitude scale
      |q w| max|E| sum|v_x| (sums of terms of both signs);
    * explicit schemes: the node charges after the step bit-exact against
      the oracle's assignment of the GPU's own new state, and the new field,
      potential, field energy and averaged profiles within 1e-9 of scale
      (the new positions themselves are compared per particle elsewhere: an
      FP32 and an FP64 push may put a particle on either side of a 2^-16
      quantisation boundary);
    * direct implicit: the predicted positions are FP32 on the GPU and FP64
      in the oracle, so about 1 % of them (those within two FP32 ulps of a
      2^-16 boundary) may take the neighbouring quantisation code: each moves
      a node charge by at most 2^19 units (2^-14 of a particle) and the
      susceptibility of a cell by at most one 2^-16 quantum; the bars are the
      summed node-charge change below 1e-5 of the total (about 60x the
      expected 1.2e-6), chi within 1e-5 relative, and the field change within
      the charge change times e w / eps0 (Gauss's law) plus 1e-9 of scale;
    * the EEDF within a few particles that FP32 and FP64 bin differently.
    The measured error of every diagnostic is printed (one line, prefix
    "diagnostic errors") and returned as the third value."""
    d0 = gpu.diag()
    scheme = cfg.get("scheme", "ec_explicit")
    implicit = scheme in ("ec_implicit", "mc_implicit")
    st = [gpu.get_particles(sp) for sp in ("e", "i")]
    # the GPU re-enters its own state at this step, so both sides draw every
    # particle's wait to its next null-collision selection alike (the waits
    # are state that the particle read-back leaves out)
    for k, sp in enumerate(("e", "i")):
        gpu.set_particles(sp, dict(st[k], abar=st[k]["abar"] if implicit else None), next_id=st[k]["next_id"])
    gpu.init_field(set_abar=False)
    orc = _oracle_of(cfg, st, d0["step"], implicit)
    g_pre = gpu.grids()
    if not implicit:  # the field the push uses is that of the state
        assert np.array_equal(g_pre["rho_q_e"], orc.grids()["rho_q_e"])
        assert np.array_equal(g_pre["rho_q_i"], orc.grids()["rho_q_i"])
    gpu.diag(reset_avg=True)
    orc.reset_averages()
    w0 = (np.array(d0["wall_count"]), np.array(d0["wall_energy_ev"]), np.array(d0["coll"]), d0["births"])
    do0 = orc.diag()
    gpu.step(1)
    orc.step(1)
    dg, do = gpu.diag(), orc.diag()
    assert dg["count"] == do["count"]
    assert (np.array(dg["wall_count"]) - w0[0]).tolist() == (np.array(do["wall_count"]) - np.array(do0["wall_count"])).tolist()
    assert (np.array(dg["coll"]) - w0[2]).tolist() == (np.array(do["coll"]) - np.array(do0["coll"])).tolist()
    assert dg["births"] - w0[3] == do["births"] - do0["births"]
    we_g = np.array(dg["wall_energy_ev"]) - w0[1]
    we_o = np.array(do["wall_energy_ev"]) - np.array(do0["wall_energy_ev"])
    np.testing.assert_allclose(we_g, we_o, rtol=1e-5, atol=1e-9)
    errs = {"wall_energy": _rel(we_g, we_o)}
    for k, sp in enumerate(("e", "i")):
        errs["ke_x_" + sp] = _rel(dg["ke_x"][k], do["ke_x"][k])
        errs["ke_perp_" + sp] = _rel(dg["ke_perp"][k], do["ke_perp"][k])
    for k in range(2):
        assert dg["ke_x"][k] == pytest.approx(do["ke_x"][k], rel=1e-5, abs=1e-30)
        assert dg["ke_perp"][k] == pytest.approx(do["ke_perp"][k], rel=1e-5, abs=1e-30)
    der = oracle.derive(cfg)
    emax = float(np.abs(g_pre["e_cc"]).max())
    for k, sp in enumerate(("e", "i")):
        scale = abs(der["q"][k]) * der["weight"] * emax * float(np.abs(st[k]["vx"].astype(np.float64)).sum())
        assert abs(dg["power"][k] - do["power"][k]) <= 1e-5 * scale + 1e-30, (sp, dg["power"][k], do["power"][k])
        errs["power_" + sp + "_of_scale"] = abs(dg["power"][k] - do["power"][k]) / max(scale, 1e-300)
    g1, pg = gpu.grids(), gpu.profiles()
    if not implicit:
        assert dg["field_energy_push"] == pytest.approx(do["field_energy_push"], rel=1e-9, abs=1e-30)
        post = [gpu.get_particles(sp) for sp in ("e", "i")]
        o2 = _oracle_of(cfg, post, dg["step"], False)
        o1 = o2.grids()
        assert np.array_equal(g1["rho_q_e"], o1["rho_q_e"]) and np.array_equal(g1["rho_q_i"], o1["rho_q_i"])
        e_tol = 1e-9 * max(np.abs(o1["e_cc"]).max(), 1e-300)
        np.testing.assert_allclose(g1["e_cc"], o1["e_cc"], rtol=0, atol=e_tol)
        np.testing.assert_allclose(g1["phi"], o1["phi"], rtol=0, atol=1e-9 * max(np.abs(o1["phi"]).max(), 1e-300))
        assert dg["field_energy"] == pytest.approx(o2.diag()["field_energy"], rel=1e-8, abs=1e-30)
        errs["field_energy_push"] = _rel(dg["field_energy_push"], do["field_energy_push"])
        errs["field_energy"] = _rel(dg["field_energy"], o2.diag()["field_energy"])
        errs["e_cc_of_scale"] = _of_scale(g1["e_cc"], o1["e_cc"])
        errs["phi_of_scale"] = _of_scale(g1["phi"], o1["phi"])
        errs["phi_avg_of_scale"] = _of_scale(pg["phi"], o1["phi"])
        # one step's averages: the potential and densities of the new field
        np.testing.assert_allclose(pg["phi"], o1["phi"], rtol=0, atol=1e-9 * max(np.abs(o1["phi"]).max(), 1e-300))
        unit = der["weight"] / node_lengths(cfg, der["dx"]) / oracle.charge_unit(cfg)
        for key, q in (("ne", o1["rho_q_e"]), ("ni", o1["rho_q_i"])):
            ref = q.astype(np.float64) * unit
            np.testing.assert_allclose(pg[key], ref, rtol=1e-12, atol=1e-12 * max(np.abs(ref).max(), 1e-300))
            errs[key + "_of_scale"] = _of_scale(pg[key], ref)
    else:
        o1 = orc.grids()
        unit = oracle.charge_unit(cfg)
        n_tot = [len(x["id"]) for x in st]
        for k, key in enumerate(("rho_q_e", "rho_q_i")):
            moved = np.abs(g1[key] - o1[key]).sum()
            assert moved <= 1e-5 * max(n_tot[k], 1) * unit, (key, moved / (max(n_tot[k], 1) * unit))
            errs[key + "_moved_of_total"] = float(moved / (max(n_tot[k], 1) * unit))
        moved_q = np.abs((g1["rho_q_i"] - g1["rho_q_e"]) - (o1["rho_q_i"] - o1["rho_q_e"])).sum()
        de = 2.0 * 1.602176634e-19 * der["weight"] / 8.8541878128e-12 * moved_q / unit
        e_tol = de + 1e-9 * max(np.abs(o1["e_cc"]).max(), 1e-300)
        np.testing.assert_allclose(g1["e_cc"], o1["e_cc"], rtol=0, atol=e_tol)
        np.testing.assert_allclose(g1["phi"], o1["phi"], rtol=0,
                                   atol=cfg["length"] * e_tol + 1e-9 * max(np.abs(o1["phi"]).max(), 1e-300))
        np.testing.assert_allclose(g1["chi"], o1["chi"], rtol=1e-5, atol=0)
        errs["chi"] = _rel(g1["chi"], o1["chi"])
        errs["e_cc_of_scale"] = _of_scale(g1["e_cc"], o1["e_cc"])
        errs["phi_of_scale"] = _of_scale(g1["phi"], o1["phi"])
        assert np.abs(o1["chi"]).max() > 0
        hmax = float(np.max(cfg["cell_width"])) if cfg.get("cell_width") is not None else der["dx"]
        w_tol = 8.8541878128e-12 * hmax * (np.abs(o1["e_cc"]).sum() * e_tol + 0.5 * len(o1["e_cc"]) * e_tol ** 2)
        assert abs(dg["field_energy"] - do["field_energy"]) <= w_tol + 1e-9 * abs(do["field_energy"])
        errs["field_energy"] = _rel(dg["field_energy"], do["field_energy"])
    diag_step = cfg.get("diag_period", 0) > 0 and d0["step"] % cfg["diag_period"] == 0
    if diag_step:
        po = orc.averages()
        cw = np.asarray(cfg["cell_width"]) if cfg.get("cell_width") is not None else der["dx"]
        for k, key in enumerate(("heat_e", "heat_i")):
            scale = abs(der["q"][k]) * der["weight"] * emax * float(np.abs(st[k]["vx"].astype(np.float64)).sum())
            dev = float((np.abs(pg[key] - po[key]) * cw).sum())
            assert dev <= 1e-5 * scale + 1e-30, key
            errs[key + "_of_scale"] = dev / max(scale, 1e-300)
        if cfg.get("eedf_bins", 0) > 0:
            diff = np.abs(pg["eedf"].astype(np.int64) - po["eedf"].astype(np.int64)).sum()
            assert diff <= (eedf_tol if eedf_tol is not None else 4), diff
            errs["eedf_particles_binned_apart"] = int(diff)
    print("diagnostic errors (%s, step %d):" % (scheme, d0["step"]),
          {k: (v if isinstance(v, int) else float("%.3g" % v)) for k, v in errs.items()})
    return dg, do, errs


# ------------------------------------------------------------------ Philox
def test_philox_words_bitexact_vs_oracle():
    import torch
    from paper_1310_5284_gb300.sim import philox_fill
    for key, ctr in (((1, 0), (0, 0, 0, 0)), ((0xDEADBEEF, 17), (123456, 99, 7, 0x01020001)),
                     ((2 ** 32 - 1, 2 ** 32 - 1), (2 ** 32 - 1000, 2 ** 32 - 1, 2 ** 32 - 1, 2 ** 32 - 1))):
        n = 200_003
        out = torch.zeros(4 * n, dtype=torch.int32, device="cuda:0")
        philox_fill(key, ctr, n, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy().view(np.uint32).reshape(n, 4)
        ref = oracle.philox_stream(key, ctr, n)
        assert np.array_equal(got, ref)


# ------------------------------------------------------------------ load
def test_uniform_load_matches_oracle():
    cfg = dict(workloads.CFG_SMALL_CCP, mcc=False)
    gpu = gpu_sim(cfg)
    orc = oracle.Sim(cfg).load(cfg["np_init"], cfg["np_init"])
    for k, sp in enumerate(("e", "i")):
        a = by_id(gpu.get_particles(sp))
        b = by_id(orc.get_species(sp))
        assert np.array_equal(a["id"], np.arange(cfg["np_init"]))
        xa = a["cell"].astype(np.float64) + a["off"].astype(np.float64)
        assert np.array_equal(xa, b["xi"])  # positions are exact (24-bit offsets)
        for comp in ("vx", "vy", "vz"):
            np.testing.assert_allclose(a[comp], b[comp], rtol=2e-6, atol=2e-6 * vth(cfg, k))
    g, o = gpu.grids(), orc.grids()
    assert np.array_equal(g["rho_q_e"], o["rho_q_e"]) and np.array_equal(g["rho_q_i"], o["rho_q_i"])


def test_stretched_load_matches_oracle():
    """The load on a non-uniform grid is uniform in x: the cell by bisection
    over the node positions and the FP32 offset, both decided in FP64 from
    the same Philox word, so positions agree exactly."""
    cfg = workloads.with_stretch(dict(workloads.CFG_SMALL_CCP, mcc=False), 0.6)
    gpu = gpu_sim(cfg)
    orc = oracle.Sim(cfg).load(cfg["np_init"], cfg["np_init"])
    for k, sp in enumerate(("e", "i")):
        a = by_id(gpu.get_particles(sp))
        b = by_id(orc.get_species(sp))
        xa = a["cell"].astype(np.float64) + a["off"].astype(np.float64)
        assert np.array_equal(xa, b["xi"])
        for comp in ("vx", "vy", "vz"):
            np.testing.assert_allclose(a[comp], b[comp], rtol=2e-6, atol=2e-6 * vth(cfg, k))
    g, o = gpu.grids(), orc.grids()
    assert np.array_equal(g["rho_q_e"], o["rho_q_e"]) and np.array_equal(g["rho_q_i"], o["rho_q_i"])
    np.testing.assert_allclose(g["e_cc"], o["e_cc"], rtol=0, atol=1e-9 * np.abs(o["e_cc"]).max())


# ------------------------------------------------------------------ deposit + field
DEPOSIT_CASES = [
    ("ec_dirichlet_64", dict(n_cells=64), 12_800, False),
    ("ec_dirichlet_ragged_77", dict(n_cells=77), 12_345, False),
    ("ec_periodic_100", dict(n_cells=100, periodic=True, rf_volt=0.0), 10_007, False),
    ("ec_dirichlet_1024_sorted", dict(n_cells=1024), 300_001, True),
    ("mc_dirichlet_64", dict(n_cells=64, scheme="mc_explicit"), 9_999, False),
    ("mc_periodic_33", dict(n_cells=33, periodic=True, scheme="mc_explicit", rf_volt=0.0), 4_321, False),
    ("mc_implicit_dirichlet_45", dict(n_cells=45, scheme="mc_implicit"), 7_777, False),
    ("ec_tiny_2cells", dict(n_cells=2), 5, False),
    ("ec3_dirichlet_64", dict(n_cells=64, scheme="ec3_explicit"), 12_800, False),
    ("ec3_periodic_100", dict(n_cells=100, periodic=True, rf_volt=0.0, scheme="ec3_explicit"), 10_007, False),
    ("ec3_dirichlet_1024_sorted", dict(n_cells=1024, scheme="ec3_explicit"), 300_001, True),
    ("ec3_periodic_3", dict(n_cells=3, periodic=True, rf_volt=0.0, scheme="ec3_explicit"), 1_001, False),
    ("ec3_tiny_2cells", dict(n_cells=2, scheme="ec3_explicit"), 5, False),
    # non-uniform grids (cells (1 -/+ beta) L/N at the electrodes / mid-gap)
    ("nu_dirichlet_64_b06", dict(n_cells=64, grid_beta=0.6), 12_800, False),
    ("nu_periodic_100_b05", dict(n_cells=100, periodic=True, rf_volt=0.0, grid_beta=0.5), 10_007, False),
    ("nu_dirichlet_1024_sorted_b07", dict(n_cells=1024, grid_beta=0.7), 300_001, True),
    ("nu_tiny_2cells", dict(n_cells=2, cell_width=[0.006, 0.014]), 5, False),
    ("nu_ec3_dirichlet_64_b06", dict(n_cells=64, scheme="ec3_explicit", grid_beta=0.6), 12_800, False),
    ("nu_ec3_periodic_100_b05", dict(n_cells=100, periodic=True, rf_volt=0.0, scheme="ec3_explicit", grid_beta=0.5),
     10_007, False),
]


@pytest.mark.parametrize("name,over,n,srt", DEPOSIT_CASES, ids=[c[0] for c in DEPOSIT_CASES])
def test_deposit_bitexact_and_field(name, over, n, srt):
    cfg = dict(workloads.CFG_SMALL_CCP, mcc=False, np_init=n)
    cfg.update(over)
    cfg = with_grid(cfg)
    gpu = gpu_sim(cfg)
    orc = oracle.Sim(cfg, cap_e=n + 16, cap_i=n + 16)
    inject(gpu, orc, cfg, states_for(cfg, n, 100 + n, sorted_cells=srt), step=37)
    g, o = gpu.grids(), orc.grids()
    assert np.array_equal(g["rho_q_e"], o["rho_q_e"]), name
    assert np.array_equal(g["rho_q_i"], o["rho_q_i"]), name
    unit = 6 * 2 ** 36 if cfg.get("scheme") == "ec3_explicit" else 2 ** 33  # one particle's charge
    assert g["rho_q_e"].sum() == n * unit and g["rho_q_i"].sum() == n * unit
    scale = max(np.abs(o["e_cc"]).max(), 1e-300)
    np.testing.assert_allclose(g["e_cc"], o["e_cc"], rtol=0, atol=1e-9 * scale)
    pscale = max(np.abs(o["phi"]).max(), 1e-300)
    np.testing.assert_allclose(g["phi"], o["phi"], rtol=0, atol=1e-9 * pscale)


def test_empty_species_and_frozen_ion_background():
    cfg = workloads.cfg_periodic(n_cells=64, np_e=5000, n0=1e15, length=0.02, dt=5e-11)
    gpu = gpu_sim(cfg)
    orc = oracle.Sim(cfg, cap_e=6000, cap_i=16)
    st = states_for(cfg, 5000, 7, ions=False)
    inject(gpu, orc, cfg, st)
    g, o = gpu.grids(), orc.grids()
    assert np.array_equal(g["rho_q_e"], o["rho_q_e"])
    assert not g["rho_q_i"].any()
    np.testing.assert_allclose(g["e_cc"], o["e_cc"], atol=1e-9 * np.abs(o["e_cc"]).max())
    # Dirichlet with a frozen ion density (the sheath case of the adjoint workload)
    cfg2 = dict(workloads.CFG_SMALL_CCP, mcc=False, ions_mobile=False, bg_density=2e15, np_init=5000)
    gpu2 = gpu_sim(cfg2)
    orc2 = oracle.Sim(cfg2, cap_e=6000, cap_i=16)
    inject(gpu2, orc2, cfg2, [st[0], None])
    g2, o2 = gpu2.grids(), orc2.grids()
    np.testing.assert_allclose(g2["phi"], o2["phi"], atol=1e-9 * np.abs(o2["phi"]).max())


# ------------------------------------------------------------------ whole steps
# (name, overrides, steps with the strict per-particle bar, total steps)
STEP_CASES = [
    ("ec_periodic_collisionless", dict(n_cells=64, periodic=True, mcc=False, rf_volt=0.0), 30, 100),
    ("ec_electrodes_rf_collisionless", dict(n_cells=64, mcc=False), 30, 100),
    ("mc_electrodes_rf_collisionless", dict(n_cells=64, mcc=False, scheme="mc_explicit"), 30, 100),
    ("ec_implicit_electrodes", dict(n_cells=64, mcc=False, scheme="ec_implicit", dt=8e-10), 5, 30),
    ("ec_implicit_periodic", dict(n_cells=50, periodic=True, mcc=False, rf_volt=0.0,
                                  scheme="ec_implicit", dt=8e-10), 10, 100),
    ("mc_implicit_electrodes", dict(n_cells=64, mcc=False, scheme="mc_implicit", dt=8e-10), 5, 30),
    ("mc_implicit_periodic", dict(n_cells=50, periodic=True, mcc=False, rf_volt=0.0,
                                  scheme="mc_implicit", dt=8e-10), 10, 100),
    ("mc_implicit_ragged_37", dict(n_cells=37, mcc=False, scheme="mc_implicit", dt=3e-10), 10, 40),
    ("ec3_periodic_collisionless", dict(n_cells=64, periodic=True, mcc=False, rf_volt=0.0,
                                        scheme="ec3_explicit"), 30, 100),
    ("ec3_electrodes_rf_collisionless", dict(n_cells=64, mcc=False, scheme="ec3_explicit"), 30, 100),
    ("ec3_ragged_37", dict(n_cells=37, mcc=False, scheme="ec3_explicit"), 30, 60),
    ("nu_periodic_collisionless_b06", dict(n_cells=64, periodic=True, mcc=False, rf_volt=0.0, grid_beta=0.6),
     30, 100),
    ("nu_electrodes_rf_collisionless_b06", dict(n_cells=64, mcc=False, grid_beta=0.6), 30, 100),
    ("nu_ragged_37_b08", dict(n_cells=37, mcc=False, grid_beta=0.8), 30, 60),
    # the largest grid the library takes: the width table beside the largest
    # accumulators in shared memory
    ("nu_1024_cells_b07", dict(n_cells=1024, np_init=40_000, mcc=False, grid_beta=0.7), 10, 30),
    ("nu_implicit_electrodes_b06", dict(n_cells=64, mcc=False, scheme="ec_implicit", dt=8e-10, grid_beta=0.6), 5, 30),
    ("nu_implicit_periodic_b05", dict(n_cells=50, periodic=True, mcc=False, rf_volt=0.0, scheme="ec_implicit",
                                      dt=8e-10, grid_beta=0.5), 10, 100),
    ("nu_ec3_electrodes_b06", dict(n_cells=64, mcc=False, scheme="ec3_explicit", grid_beta=0.6), 30, 100),
    ("nu_ec3_periodic_b05", dict(n_cells=64, periodic=True, mcc=False, rf_volt=0.0, scheme="ec3_explicit",
                                 grid_beta=0.5), 30, 100),
]


@pytest.mark.parametrize("name,over,strict,steps", STEP_CASES, ids=[c[0] for c in STEP_CASES])
def test_steps_match_oracle(name, over, strict, steps):
    """Collisionless steps from a seeded state.  Over the first `strict` steps
    every particle is within 1e-5 (of L for positions, of max(|v|, v_th) for
    velocities): there the FP64 oracle itself, with its state rounded to FP32
    after every step, stays 8-100x inside that bar.  Beyond, the plasma's
    chaos amplifies FP32 rounding (the implicit runs at omega_p dt = 2 most):
    the GPU's divergence must then be no worse than 4x the oracle's own
    divergence under FP32 rounding (99th percentile and maximum)."""
    cfg = dict(workloads.CFG_SMALL_CCP, np_init=12_800, sort_period=8)
    cfg.update(over)
    cfg = with_grid(cfg)
    n = cfg["np_init"]
    gpu = gpu_sim(cfg)
    orc = oracle.Sim(cfg)
    states = states_for(cfg, n, 5 + len(name))
    inject(gpu, orc, cfg, states)
    g0 = gpu.grids()
    assert np.array_equal(g0["rho_q_e"], orc.grids()["rho_q_e"])
    gpu.step(strict)
    orc.step(strict)
    if cfg.get("cell_width") is None:
        compare_particles(gpu, orc, cfg)
    else:
        # on a non-uniform grid the force jumps at a node where the cell width
        # changes (by the width ratio, up to 6 % here), so a particle that FP32
        # and FP64 put on either side of a node in a strong field diverges from
        # the first steps: the bar is the oracle's own FP32 sensitivity
        compare_particles(gpu, orc, cfg, floor=fp32_sensitivity(cfg, states, strict))
    gpu.step(steps - strict)
    orc.step(steps - strict)
    assert gpu.status() == 0  # no capacity, birth-buffer or bounded-wait flag
    dg, do = gpu.diag(), orc.diag()
    assert dg["step"] == do["step"] == steps
    floor = fp32_sensitivity(cfg, states, steps)
    if all(f is not None and f["same_set"] for f in floor):
        assert dg["count"] == do["count"], name
        assert dg["wall_count"] == do["wall_count"], name
        compare_particles(gpu, orc, cfg, floor=floor)
        # the kinetic energy follows from the per-particle bar (ke_bar); the
        # field energy of a noisy 64-cell plasma is checked where chaos plays
        # no part, in the one-step comparison below
        for k in range(2):
            assert abs(dg["ke_x"][k] - do["ke_x"][k]) <= ke_bar(1e-5, floor[k]) * abs(do["ke_x"][k]) + 1e-30
    else:
        # FP32 rounding alone changes which particles reach an electrode: the
        # counts may differ by the decisions rounding flips, a few at most
        for k in range(2):
            assert abs(dg["count"][k] - do["count"][k]) <= 8
    one_step_diagnostics(gpu, cfg)


IMPLICIT_GRID_CASES = [
    ("ec_implicit_electrodes_64", dict(n_cells=64, scheme="ec_implicit", dt=8e-10)),
    ("ec_implicit_periodic_50", dict(n_cells=50, periodic=True, rf_volt=0.0, scheme="ec_implicit", dt=8e-10)),
    ("mc_implicit_electrodes_45", dict(n_cells=45, scheme="mc_implicit", dt=3e-10)),
    ("mc_implicit_periodic_33", dict(n_cells=33, periodic=True, rf_volt=0.0, scheme="mc_implicit", dt=8e-10)),
    ("nu_implicit_electrodes_64_b06", dict(n_cells=64, scheme="ec_implicit", dt=8e-10, grid_beta=0.6)),
    ("nu_implicit_periodic_50_b05", dict(n_cells=50, periodic=True, rf_volt=0.0, scheme="ec_implicit", dt=8e-10,
                                         grid_beta=0.5)),
]


@pytest.mark.parametrize("name,over", IMPLICIT_GRID_CASES, ids=[c[0] for c in IMPLICIT_GRID_CASES])
def test_implicit_susceptibility_and_modified_poisson_grid(name, over):
    """Direct-implicit steps from a seeded state with a given abar: the
    susceptibility the predictor assigns, the node charges of the predicted
    positions, and the potential and field of the modified Poisson equation
    grid point by grid point against the oracle, with every other diagnostic
    of the step (one_step_diagnostics; the bars follow from the FP32
    predictor's quantisation decisions)."""
    cfg = dict(workloads.CFG_SMALL_CCP, np_init=12_800, sort_period=4, diag_period=1, eedf_bins=30)
    cfg.update(over)
    cfg = with_grid(cfg)
    n = cfg["np_init"]
    gpu = gpu_sim(cfg)
    orc = oracle.Sim(cfg)
    states = states_for(cfg, n, 300 + cfg["n_cells"])
    rng = np.random.default_rng(cfg["n_cells"])
    qm = [-E / ME, E / (cfg.get("ion_mass_amu", 39.948) * AMU)]
    abar = [np.float32(0.3 * qm[k] * 1e3) * rng.standard_normal(n).astype(np.float32) for k in range(2)]
    inject(gpu, orc, cfg, states, step=7, abar=abar)
    # the first step's predictor: its positions differ from the oracle's only
    # by FP32 rounding of two products (see one_step_diagnostics for the bar)
    gpu.step(1)
    orc.step(1)
    g, o = gpu.grids(), orc.grids()
    assert np.abs(o["chi"]).max() > 0
    np.testing.assert_allclose(g["chi"], o["chi"], rtol=1e-5, atol=0)
    one_step_diagnostics(gpu, cfg, eedf_tol=4)


COLLISION_CASES = [
    ("ec_explicit", {}), ("ec_implicit", {}), ("mc_implicit", {}), ("ec3_explicit", {}),
    # the collision-model options: Opal-Pollock-Wagner split, Vahedi-Surendra scattering
    ("ec_explicit", dict(iz_split="opal")),
    ("ec_explicit", dict(scattering="vahedi_surendra")),
    ("ec_implicit", dict(iz_split="opal", scattering="vahedi_surendra", te_ev=10.0)),
    ("ec_explicit", dict(grid_beta=0.6)),  # non-uniform grid
    ("ec_explicit", dict(grid_beta=0.5, periodic=True, rf_volt=0.0)),  # non-uniform periodic box
    ("ec_implicit", dict(grid_beta=0.6)),  # direct implicit on a non-uniform grid
    ("ec3_explicit", dict(grid_beta=0.6)),  # m = 3 on a non-uniform grid
]


@pytest.mark.parametrize("scheme,opts", COLLISION_CASES,
                         ids=["%s%s" % (c[0], "".join("-" + str(v) for v in c[1].values())) for c in COLLISION_CASES])
def test_collisions_counts_exact_and_births_ranked(scheme, opts):
    """Null-collision MCC on the same Philox stream: selection is an integer
    compare, so tallies and births agree exactly; children get the same ids
    (and, in the implicit schemes, the parent's abar)."""
    cfg = dict(workloads.CFG_SMALL_CCP, np_init=20_000, sort_period=4, te_ev=6.0, scheme=scheme,
               diag_period=1, eedf_bins=40)
    cfg.update(opts)
    cfg = with_grid(cfg)
    n = cfg["np_init"]
    gpu = gpu_sim(cfg)
    orc = oracle.Sim(cfg)
    states = states_for(cfg, n, 77)
    inject(gpu, orc, cfg, states, step=1000)
    for _ in range(4):
        gpu.step(5)
        orc.step(5)
    dg, do = gpu.diag(), orc.diag()
    assert dg["coll"] == do["coll"]
    assert dg["births"] == do["births"] > 0
    assert dg["count"] == do["count"]
    assert dg["wall_count"] == do["wall_count"]
    assert dg["overflow"] == do["overflow"]
    # The collision kinematics amplify rounding near a threshold (the speed
    # after excitation or ionisation is sqrt(eps - threshold)); the bar is the
    # one of the collisionless runs: 1e-5, or 4x the oracle's own divergence
    # when its state is rounded to FP32 after every step, over the same steps
    # and Philox streams.
    floor = fp32_sensitivity(cfg, states, 20, step0=1000)
    compare_particles(gpu, orc, cfg, floor=floor)
    if scheme in ("ec_implicit", "mc_implicit"):  # abar of parents and children, relative to its scale
        for k, sp in enumerate(("e", "i")):
            a, b = by_id(gpu.get_particles(sp)), by_id(orc.get_species(sp))
            d = np.abs(a["abar"].astype(np.float64) - b["abar"]) / np.abs(b["abar"]).max()
            assert d.max() <= max(1e-5, floor[k]["abar"]), (sp, d.max(), floor[k]["abar"])
    one_step_diagnostics(gpu, cfg, eedf_tol=8)


@pytest.mark.parametrize("n", [40_000, 120_000])
def test_many_births_per_step_ranked_like_oracle(n):
    """Hot electrons (40 eV) ionise about 2 % of themselves per step, so one
    step records hundreds to thousands of births: the ranking by parent id
    goes through the bucketed paths (in shared memory up to 1024 births, in
    global memory beyond) and must still hand out the oracle's ids."""
    cfg = dict(workloads.CFG_SMALL_CCP, np_init=n, sort_period=4, te_ev=40.0,
               births_capacity=8192)
    gpu = gpu_sim(cfg)
    orc = oracle.Sim(cfg)
    states = states_for(cfg, n, 91)
    inject(gpu, orc, cfg, states, step=500)
    for _ in range(3):
        gpu.step(1)
        orc.step(1)
    dg, do = gpu.diag(), orc.diag()
    assert gpu.status() == 0
    assert dg["births"] == do["births"] > 3 * (300 if n < 100_000 else 1100)
    assert dg["coll"] == do["coll"]
    assert dg["count"] == do["count"]
    compare_particles(gpu, orc, cfg, floor=fp32_sensitivity(cfg, states, 3, step0=500))


@pytest.mark.parametrize("scheme", ["ec_explicit", "ec3_explicit", "nu"])
def test_sorting_and_graph_replay_do_not_change_results(scheme):
    """Charge sums are integers and draws are keyed on (id, step), so the
    slot order (sorted or not) and graph replay leave every particle
    bit-identical (nu: the explicit EC scheme on a stretched grid)."""
    if scheme == "nu":
        base = workloads.with_stretch(dict(workloads.CFG_SMALL_CCP, np_init=12_800), 0.6)
    else:
        base = dict(workloads.CFG_SMALL_CCP, np_init=12_800, scheme=scheme)
    outs = []
    for sp in (0, 1, 16):
        cfg = dict(base, sort_period=sp)
        gpu = gpu_sim(cfg)
        gpu.step(48)
        outs.append({s: by_id(gpu.get_particles(s)) for s in ("e", "i")})
        gpu.close()
    for s in ("e", "i"):
        for o in outs[1:]:
            for key in ("id", "cell", "off", "vx", "vy", "vz"):
                assert np.array_equal(o[s][key], outs[0][s][key]), (s, key)


@pytest.mark.parametrize("beta", [None, 0.6])
def test_checkpoint_resume_is_bit_identical(beta):
    """A snapshot restores the run exactly (beta: on a stretched grid, whose
    width tables travel in the arena)."""
    cfg = dict(workloads.CFG_SMALL_CCP, np_init=8000, sort_period=4)
    if beta is not None:
        cfg = workloads.with_stretch(cfg, beta)
    gpu = gpu_sim(cfg)
    gpu.step(20)
    snap = gpu.save()
    gpu.step(30)
    ref = {s: by_id(gpu.get_particles(s)) for s in ("e", "i")}
    ref_diag = gpu.diag()
    gpu.load(snap)
    gpu.step(30)
    got = {s: by_id(gpu.get_particles(s)) for s in ("e", "i")}
    for s in ("e", "i"):
        for key in ("id", "cell", "off", "vx", "vy", "vz"):
            assert np.array_equal(got[s][key], ref[s][key])
    d = gpu.diag()
    assert d["coll"] == ref_diag["coll"] and d["count"] == ref_diag["count"]


def test_birth_capacity_overflow_sets_status_without_fault():
    cfg = dict(workloads.CFG_SMALL_CCP, np_init=20_000, te_ev=8.0, births_capacity=2)
    gpu = gpu_sim(cfg)
    gpu.step(20)
    assert gpu.status() & 0x2
    d = gpu.diag()
    assert d["count"][0] == d["count"][1] + (d["count"][0] - d["count"][1])  # readable after overflow


def test_handles_of_different_sizes_coexist():
    """A large run created before a small one still steps afterwards: each
    launch's shared-memory request stays within the kernel's limit, which
    only rises."""
    big = gpu_sim(dict(workloads.CFG_SMALL_CCP, n_cells=1024, np_init=20_000, eedf_bins=1024))
    small = gpu_sim(dict(workloads.CFG_SMALL_CCP, n_cells=16, np_init=2_000, eedf_bins=8))
    big.step(3)
    small.step(3)
    big.init_field()
    assert big.diag()["step"] == 3 and small.diag()["step"] == 3
    assert big.status() == 0 and small.status() == 0
    big.close()
    small.close()


@pytest.mark.parametrize("bad", ["cell_low", "cell_high", "offset_one", "offset_nan"])
def test_set_particles_rejects_off_grid_and_applies_nothing(bad):
    """The upload is checked on the device; a particle off the grid makes the
    call fail and leaves the run's particles as they were."""
    from paper_1310_5284_gb300._abi import PicError

    cfg = dict(workloads.CFG_SMALL_CCP, mcc=False, np_init=5000)
    gpu = gpu_sim(cfg)
    before = by_id(gpu.get_particles("e"))
    st = workloads.injected_particles(3, 4000, cfg["n_cells"], vth(cfg, 0))
    k = 3999 if bad != "cell_low" else 1234
    if bad == "cell_low":
        st["cell"][k] = -1
    elif bad == "cell_high":
        st["cell"][k] = cfg["n_cells"]
    elif bad == "offset_one":
        st["off"][k] = 1.0
    else:
        st["off"][k] = np.nan
    with pytest.raises(PicError, match="particle %d outside the grid" % k):
        gpu.set_particles("e", st)
    after = by_id(gpu.get_particles("e"))
    for key in ("id", "cell", "off", "vx", "vy", "vz"):
        assert np.array_equal(before[key], after[key]), key
    st["off"][k] = 0.5
    st["cell"][k] = 3
    gpu.set_particles("e", st)  # the corrected upload goes through
    assert gpu.get_particles("e")["id"].size == 4000
    gpu.close()


@pytest.mark.parametrize("scheme", ["ec_explicit", "ec_implicit"])
def test_set_state_is_both_uploads_in_one_call(scheme):
    """pic_set_state gives the run exactly what two pic_set_particles calls
    give (every particle after ten steps), and a particle off the grid in
    either species leaves both species as they were."""
    from paper_1310_5284_gb300._abi import PicError

    cfg = dict(workloads.CFG_SMALL_CCP, np_init=6000, scheme=scheme)
    st = states_for(cfg, 5000, 21)
    if scheme == "ec_implicit":
        rng = np.random.default_rng(5)
        for s in st:
            s["abar"] = rng.normal(size=len(s["id"])).astype(np.float32) * 1e12
    a, b = gpu_sim(cfg), gpu_sim(cfg)
    a.set_particles("e", st[0])
    a.set_particles("i", st[1])
    b.set_state(st[0], st[1])
    for g in (a, b):
        g.set_step(11)
        g.init_field(set_abar=False)
        g.step(10)
    for sp in ("e", "i"):
        pa, pb = by_id(a.get_particles(sp)), by_id(b.get_particles(sp))
        for key in ("id", "cell", "off", "vx", "vy", "vz", "abar"):
            assert np.array_equal(pa[key], pb[key]), (sp, key)
    before = {sp: by_id(b.get_particles(sp)) for sp in ("e", "i")}
    bad = {k: v.copy() for k, v in st[1].items()}
    bad["cell"][77] = cfg["n_cells"]
    with pytest.raises(PicError, match="particle 77 outside the grid"):
        b.set_state(st[0], bad)
    for sp in ("e", "i"):
        after = by_id(b.get_particles(sp))
        for key in ("id", "cell", "off", "vx", "vy", "vz"):
            assert np.array_equal(before[sp][key], after[key]), (sp, key)
    a.close()
    b.close()


def test_high_selection_implicit_run_keeps_the_drain_in_step():
    """A direct-implicit discharge at omega_p dt = 2 selects about a third of
    its particles for a collision every step, so the collision queue crosses
    its drain mark in the middle of a block's stream many times per launch.
    The drain decision must be the same in every thread of a block (a block
    whose warps disagreed entered different barriers and faulted the GPU on
    exactly this configuration, run 47 of the batched sweep).  Bar: fifteen
    steps through the single-run path (one sort among them) end with a clean
    status word, particle counts conserved by the tallies, and the same
    particles as a second run of the same configuration."""

    spec = dict(workloads.batch_configs(256)[47], omega_p_dt=2.0)  # the run's step when it faulted
    cfg = workloads.discharge_from_spec(spec)
    assert cfg["scheme"] == "ec_implicit" and cfg["np_init"] > 1_500_000
    runs = []
    for _ in range(2):
        gpu = gpu_sim(cfg)
        gpu.step(15)
        d = gpu.diag()
        assert gpu.status() == 0
        assert d["step"] == 15
        assert sum(d["coll"]) > 0.05 * 15 * cfg["np_init"]  # selections, real and null
        born = d["births"]
        lost = [d["wall_count"][k][0] + d["wall_count"][k][1] for k in range(2)]
        for k in range(2):
            assert d["count"][k] == cfg["np_init"] + born - lost[k]
        runs.append(by_id(gpu.get_particles("e")))
        gpu.close()
    for key in ("id", "cell", "off", "vx", "vy", "vz"):
        assert np.array_equal(runs[0][key], runs[1][key]), key
