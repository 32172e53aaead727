"""Plain FP64 CPU oracle for the 1D electrostatic PIC/MCC method of Wang, Sun,
Jiang & Kong (energy-conserving PIC/MC benchmarked on RF discharges).

TEST INFRASTRUCTURE ONLY.  This package is imported by the tests, by the smoke
check and by the CPU-baseline leg of the benchmark; the product library never
imports, links or calls it, and it shares no code with the CUDA path.  The
arithmetic lives in ``oracle.c`` (compiled with gcc on first use, or by the
repository's build step); this module only marshals numpy arrays.

Every function cites the passage of the paper it follows in ``oracle.c``:
Eq. (2) charge assignment, Eq. (3) force interpolation, Sec. 2 schemes (1)-(4),
Sec. 3 discharge model (electrodes, absorption, collisions, uniform load).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_SRC_ADJ = os.path.join(_HERE, "adjoint.c")
_HDR = os.path.join(_HERE, "oracle.h")
_SO = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

SCHEMES = {"ec_explicit": 0, "mc_explicit": 1, "ec_implicit": 2, "mc_implicit": 3, "ec3_explicit": 4}
SPECIES = {"e": 0, "i": 1}

# conversion of a gas pressure to a density is part of the workload description
_TORR_PA = 101325.0 / 760.0
_KB = 1.380649e-23


def build(force: bool = False) -> str:
    """Compile liboracle.so next to its source (plain C, IEEE FP64, no contraction)."""
    with _lock:
        stale = (not os.path.exists(_SO)) or any(
            os.path.getmtime(f) > os.path.getmtime(_SO) for f in (_SRC, _SRC_ADJ, _HDR))
        if force or stale:
            tmp = _SO + ".tmp.%d" % os.getpid()
            subprocess.check_call(
                ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
                 "-fno-fast-math", _SRC, _SRC_ADJ, "-o", tmp, "-lm"])
            os.replace(tmp, _SO)
    return _SO


class Params(ctypes.Structure):
    _fields_ = [
        ("n_cells", ctypes.c_int32), ("periodic", ctypes.c_int32),
        ("scheme", ctypes.c_int32), ("mcc", ctypes.c_int32),
        ("ions_mobile", ctypes.c_int32), ("quantized", ctypes.c_int32),
        ("diag_period", ctypes.c_int32), ("eedf_bins", ctypes.c_int32),
        ("seed", ctypes.c_uint32), ("run", ctypes.c_uint32),
        ("length", ctypes.c_double), ("dt", ctypes.c_double),
        ("rf_freq", ctypes.c_double), ("rf_volt", ctypes.c_double),
        ("n0", ctypes.c_double), ("np_init", ctypes.c_double),
        ("bg_density", ctypes.c_double),
        ("te_ev", ctypes.c_double), ("ti_ev", ctypes.c_double),
        ("ion_mass_amu", ctypes.c_double),
        ("gas_density", ctypes.c_double), ("gas_temp", ctypes.c_double),
        ("sig_el", ctypes.c_double), ("exc_thr", ctypes.c_double),
        ("exc_ramp_end", ctypes.c_double), ("sig_exc_max", ctypes.c_double),
        ("iz_thr", ctypes.c_double), ("sig_iz_peak", ctypes.c_double),
        ("sig_cx", ctypes.c_double), ("eps_cap", ctypes.c_double),
        ("cx_vmax", ctypes.c_double), ("eedf_max_ev", ctypes.c_double),
        ("coll_model", ctypes.c_int32), ("reserved", ctypes.c_int32), ("iz_split_b", ctypes.c_double),
        ("cell_width", ctypes.POINTER(ctypes.c_double)),
    ]


class Derived(ctypes.Structure):
    _fields_ = [
        ("dx", ctypes.c_double), ("weight", ctypes.c_double),
        ("q", ctypes.c_double * 2), ("m", ctypes.c_double * 2),
        ("vth", ctypes.c_double * 2), ("vth_gas", ctypes.c_double),
        ("nu_max_e", ctypes.c_double), ("nu_max_i", ctypes.c_double),
        ("p_null_e", ctypes.c_double), ("p_null_i", ctypes.c_double),
        ("thr_e", ctypes.c_uint32), ("thr_i", ctypes.c_uint32),
        ("g_max_i", ctypes.c_double),
        ("wait_thr", ((ctypes.c_uint32 * 64) * 3) * 2),
    ]


class Diag(ctypes.Structure):
    _fields_ = [
        ("count", ctypes.c_int64 * 2),
        ("wall_count", (ctypes.c_int64 * 2) * 2),
        ("wall_energy_ev", (ctypes.c_double * 2) * 2),
        ("coll", ctypes.c_int64 * 5),
        ("overflow", ctypes.c_int64 * 2),
        ("births", ctypes.c_int64),
        ("ke_x", ctypes.c_double * 2),
        ("ke_perp", ctypes.c_double * 2),
        ("field_energy", ctypes.c_double),
        ("field_energy_push", ctypes.c_double),
        ("power", ctypes.c_double * 2),
        ("step", ctypes.c_int64),
        ("n_avg", ctypes.c_int64),
        ("n_diag", ctypes.c_int64),
    ]


_P = ctypes.POINTER
_d = _P(ctypes.c_double)
_i64 = _P(ctypes.c_int64)
_u32 = _P(ctypes.c_uint32)


def lib():
    global _lib
    if _lib is None:
        so = build()
        L = ctypes.CDLL(so)
        L.orc_philox4x32_10.argtypes = [_u32, _u32, _u32]
        L.orc_philox_stream.argtypes = [ctypes.c_uint32] * 6 + [ctypes.c_int64, _u32]
        L.orc_derive.argtypes = [_P(Params), _P(Derived)]
        L.orc_wait_draws.argtypes = [_P(Params), ctypes.c_int, ctypes.c_int64, _u32, ctypes.c_int64,
                                     ctypes.c_uint32, _u32]
        L.orc_deposit_s2_fixed.argtypes = [_P(Params), ctypes.c_int64, _d, _i64]
        L.orc_deposit_s2_fp64.argtypes = [_P(Params), ctypes.c_int64, _d, _d]
        L.orc_deposit_s1_fixed.argtypes = [_P(Params), ctypes.c_int64, _d, _i64]
        L.orc_deposit_s3_fixed.argtypes = [_P(Params), ctypes.c_int64, _d, _i64]
        L.orc_deposit_s3_fp64.argtypes = [_P(Params), ctypes.c_int64, _d, _d]
        L.orc_charge_unit.argtypes = [_P(Params)]
        L.orc_charge_unit.restype = ctypes.c_int64
        L.orc_gather_ec3.argtypes = [_P(Params), _d, ctypes.c_double]
        L.orc_gather_ec3.restype = ctypes.c_double
        L.orc_solve_dirichlet.argtypes = [ctypes.c_int, ctypes.c_double, _d, _d,
                                          ctypes.c_double, _d]
        L.orc_solve_periodic.argtypes = [ctypes.c_int, ctypes.c_double, _d, _d, _d]
        L.orc_fields.argtypes = [_P(Params), _d, _d, _d]
        L.orc_gather_ec.argtypes = [_P(Params), _d, ctypes.c_double]
        L.orc_gather_ec.restype = ctypes.c_double
        L.orc_gather_mc.argtypes = [_P(Params), _d, ctypes.c_double]
        L.orc_gather_mc.restype = ctypes.c_double
        L.orc_grid_nodes.argtypes = [ctypes.c_int, _d, _d]
        L.orc_locate.argtypes = [ctypes.c_int, _d, _d, ctypes.c_double, _i64, _d]
        L.orc_solve_dirichlet_h.argtypes = [ctypes.c_int, _d, _d, _d, ctypes.c_double, _d]
        L.orc_solve_periodic_h.argtypes = [ctypes.c_int, _d, _d, _d, _d]
        L.orc_gather_ec_h.argtypes = [_P(Params), _d, ctypes.c_double]
        L.orc_gather_ec_h.restype = ctypes.c_double
        L.orc_gather_ec3_h.argtypes = [_P(Params), _d, ctypes.c_double]
        L.orc_gather_ec3_h.restype = ctypes.c_double
        L.orc_rotate.argtypes = [_d, ctypes.c_double, ctypes.c_double, _d]
        L.orc_vs_cos_chi.argtypes = [ctypes.c_double, ctypes.c_double]
        L.orc_vs_cos_chi.restype = ctypes.c_double
        L.orc_opal_secondary.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double]
        L.orc_opal_secondary.restype = ctypes.c_double
        L.orc_sim_create.argtypes = [_P(Params), ctypes.c_int64, ctypes.c_int64]
        L.orc_sim_create.restype = ctypes.c_void_p
        L.orc_sim_free.argtypes = [ctypes.c_void_p]
        L.orc_sim_load.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64]
        L.orc_sim_set.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, _d, _d, _d,
                                  _d, _u32, _d, ctypes.c_uint32, _u32]
        L.orc_sim_init_field.argtypes = [ctypes.c_void_p, ctypes.c_int]
        L.orc_sim_count.argtypes = [ctypes.c_void_p, ctypes.c_int]
        L.orc_sim_count.restype = ctypes.c_int64
        L.orc_sim_get.argtypes = [ctypes.c_void_p, ctypes.c_int, _d, _d, _d, _d, _u32, _d, _u32]
        L.orc_sim_step.argtypes = [ctypes.c_void_p, ctypes.c_int64]
        L.orc_sim_set_step.argtypes = [ctypes.c_void_p, ctypes.c_int64]
        L.orc_sim_diag.argtypes = [ctypes.c_void_p, _P(Diag)]
        L.orc_sim_grids.argtypes = [ctypes.c_void_p, _i64, _i64, _d, _d, _d]
        L.orc_sim_averages.argtypes = [ctypes.c_void_p, _d, _d, _d, _d, _d, _i64]
        L.orc_sim_reset_averages.argtypes = [ctypes.c_void_p]
        L.orc_adj_forward.argtypes = [_P(AdjProblem), ctypes.c_int64, _d, _d, _d, _d, _d, _d, _i64]
        L.orc_adj_gradient.argtypes = [_P(AdjProblem), ctypes.c_int64, _d, _d, _d, _d, _d, _d]
        _lib = L
    return _lib


def _ptr(a, ct):
    if a is None:
        return None
    return a.ctypes.data_as(_P(ct))


def params(cfg: dict) -> Params:
    """Build the oracle's parameter block from a workload description dict."""
    p = Params()
    p.n_cells = int(cfg["n_cells"])
    p.periodic = int(bool(cfg.get("periodic", False)))
    p.scheme = SCHEMES[cfg.get("scheme", "ec_explicit")]
    p.mcc = int(bool(cfg.get("mcc", True)))
    p.ions_mobile = int(bool(cfg.get("ions_mobile", True)))
    p.quantized = int(bool(cfg.get("quantized", True)))
    p.diag_period = int(cfg.get("diag_period", 0))
    p.eedf_bins = int(cfg.get("eedf_bins", 100))
    p.seed = int(cfg.get("seed", 1)) & 0xffffffff
    p.run = int(cfg.get("run", 0)) & 0xffffffff
    p.length = float(cfg["length"])
    p.dt = float(cfg["dt"])
    p.rf_freq = float(cfg.get("rf_freq", 0.0))
    p.rf_volt = float(cfg.get("rf_volt", 0.0))
    p.n0 = float(cfg["n0"])
    p.np_init = float(cfg["np_init"])
    p.bg_density = float(cfg.get("bg_density", 0.0))
    p.te_ev = float(cfg.get("te_ev", 2.0))
    p.ti_ev = float(cfg.get("ti_ev", 0.026))
    p.ion_mass_amu = float(cfg.get("ion_mass_amu", 39.948))
    p.gas_temp = float(cfg.get("gas_temp", 300.0))
    p.gas_density = float(cfg.get("pressure_mtorr", 0.0)) * 1e-3 * _TORR_PA / (_KB * p.gas_temp)
    p.sig_el = float(cfg.get("sig_el", 1e-19))
    p.exc_thr = float(cfg.get("exc_thr", 11.5))
    p.exc_ramp_end = float(cfg.get("exc_ramp_end", 23.0))
    p.sig_exc_max = float(cfg.get("sig_exc_max", 5e-21))
    p.iz_thr = float(cfg.get("iz_thr", 15.8))
    p.sig_iz_peak = float(cfg.get("sig_iz_peak", 3e-20))
    p.sig_cx = float(cfg.get("sig_cx", 5e-19))
    p.eps_cap = float(cfg.get("eps_cap", 100.0))
    p.cx_vmax = float(cfg.get("cx_vmax", 2.0 * p.rf_volt + 50.0))
    p.eedf_max_ev = float(cfg.get("eedf_max_ev", 50.0))
    p.coll_model = (1 if cfg.get("iz_split", "equal") == "opal" else 0) | \
        (2 if cfg.get("scattering", "isotropic") == "vahedi_surendra" else 0)
    p.iz_split_b = float(cfg.get("iz_split_b", 10.0))
    if cfg.get("cell_width") is not None:
        h = np.ascontiguousarray(cfg["cell_width"], dtype=np.float64)
        if h.shape != (p.n_cells,) or not np.all(h > 0):
            raise ValueError("cell_width must hold n_cells positive widths")
        if abs(h.sum() - p.length) > 1e-9 * p.length:
            raise ValueError("cell widths must sum to length")
        p._cell_width = h  # keeps the array alive while the struct points at it
        p.cell_width = h.ctypes.data_as(_P(ctypes.c_double))
    return p


def derive(cfg_or_params) -> dict:
    p = cfg_or_params if isinstance(cfg_or_params, Params) else params(cfg_or_params)
    d = Derived()
    lib().orc_derive(ctypes.byref(p), ctypes.byref(d))
    return {
        "dx": d.dx, "weight": d.weight, "q": tuple(d.q), "m": tuple(d.m),
        "vth": tuple(d.vth), "vth_gas": d.vth_gas, "nu_max_e": d.nu_max_e,
        "nu_max_i": d.nu_max_i, "p_null_e": d.p_null_e, "p_null_i": d.p_null_i,
        "thr_e": d.thr_e, "thr_i": d.thr_i, "g_max_i": d.g_max_i,
        "wait_thr": np.array([[list(d.wait_thr[k][g]) for g in range(3)] for k in range(2)], dtype=np.uint64),
    }


def wait_draws(cfg, species, ids, step, sub=1) -> np.ndarray:
    """Steps to the next null-collision selection drawn for each id at `step`
    (sub 0: after a selection, 1: on entering the run); bit 30 marks a count
    that ends in a fresh draw instead of a selection."""
    p = params(cfg)
    ids = np.ascontiguousarray(ids, dtype=np.uint32)
    out = np.zeros(len(ids), dtype=np.uint32)
    lib().orc_wait_draws(ctypes.byref(p), int(SPECIES.get(species, species)), len(ids),
                         _ptr(ids, ctypes.c_uint32), int(step), int(sub), _ptr(out, ctypes.c_uint32))
    return out


def vs_cos_chi(eps_ev, u) -> np.ndarray:
    """cos chi of Vahedi-Surendra anisotropic scattering at energy eps_ev for uniforms u."""
    u = np.atleast_1d(np.asarray(u, dtype=np.float64))
    return np.array([lib().orc_vs_cos_chi(float(eps_ev), float(x)) for x in u])


def opal_secondary(excess_ev, b_ev, u) -> np.ndarray:
    """Secondary-electron energy of an ionisation (Opal-Pollock-Wagner) for uniforms u."""
    u = np.atleast_1d(np.asarray(u, dtype=np.float64))
    return np.array([lib().orc_opal_secondary(float(excess_ev), float(b_ev), float(x)) for x in u])


def philox(key, ctr) -> np.ndarray:
    k = np.ascontiguousarray(key, dtype=np.uint32)
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(_ptr(k, ctypes.c_uint32), _ptr(c, ctypes.c_uint32),
                            _ptr(out, ctypes.c_uint32))
    return out


def philox_stream(key, ctr0, n) -> np.ndarray:
    """n blocks with counter (ctr0[0] + k, ctr0[1], ctr0[2], ctr0[3]); shape (n, 4)."""
    out = np.zeros(4 * n, dtype=np.uint32)
    lib().orc_philox_stream(int(key[0]), int(key[1]), int(ctr0[0]), int(ctr0[1]),
                            int(ctr0[2]), int(ctr0[3]), int(n), _ptr(out, ctypes.c_uint32))
    return out.reshape(n, 4)


def deposit_s2_fixed(cfg, xi) -> np.ndarray:
    p = params(cfg)
    x = np.ascontiguousarray(xi, dtype=np.float64)
    out = np.zeros(p.n_cells + 1, dtype=np.int64)
    lib().orc_deposit_s2_fixed(ctypes.byref(p), len(x), _ptr(x, ctypes.c_double),
                               _ptr(out, ctypes.c_int64))
    return out


def deposit_s2_fp64(cfg, xi) -> np.ndarray:
    p = params(cfg)
    x = np.ascontiguousarray(xi, dtype=np.float64)
    out = np.zeros(p.n_cells + 1, dtype=np.float64)
    lib().orc_deposit_s2_fp64(ctypes.byref(p), len(x), _ptr(x, ctypes.c_double),
                              _ptr(out, ctypes.c_double))
    return out


def deposit_s1_fixed(cfg, xi) -> np.ndarray:
    p = params(cfg)
    x = np.ascontiguousarray(xi, dtype=np.float64)
    out = np.zeros(p.n_cells + 1, dtype=np.int64)
    lib().orc_deposit_s1_fixed(ctypes.byref(p), len(x), _ptr(x, ctypes.c_double),
                               _ptr(out, ctypes.c_int64))
    return out


def deposit_s3_fixed(cfg, xi) -> np.ndarray:
    """m = 3 assignment in units of 2^-36/6 particle charge (12-bit offset code)."""
    p = params(cfg)
    x = np.ascontiguousarray(xi, dtype=np.float64)
    out = np.zeros(p.n_cells + 1, dtype=np.int64)
    lib().orc_deposit_s3_fixed(ctypes.byref(p), len(x), _ptr(x, ctypes.c_double),
                               _ptr(out, ctypes.c_int64))
    return out


def deposit_s3_fp64(cfg, xi) -> np.ndarray:
    p = params(cfg)
    x = np.ascontiguousarray(xi, dtype=np.float64)
    out = np.zeros(p.n_cells + 1, dtype=np.float64)
    lib().orc_deposit_s3_fp64(ctypes.byref(p), len(x), _ptr(x, ctypes.c_double),
                              _ptr(out, ctypes.c_double))
    return out


def charge_unit(cfg) -> int:
    """Integer node charge of one particle charge in the scheme's fixed point."""
    p = params(cfg)
    return int(lib().orc_charge_unit(ctypes.byref(p)))


def solve_dirichlet(n_cells, dx, rho, v_left, chi=None) -> np.ndarray:
    r = np.ascontiguousarray(rho, dtype=np.float64)
    c = None if chi is None else np.ascontiguousarray(chi, dtype=np.float64)
    phi = np.zeros(n_cells + 1, dtype=np.float64)
    lib().orc_solve_dirichlet(int(n_cells), float(dx), _ptr(r, ctypes.c_double),
                              _ptr(c, ctypes.c_double), float(v_left),
                              _ptr(phi, ctypes.c_double))
    return phi


def solve_periodic(n_cells, dx, rho, chi=None) -> np.ndarray:
    r = np.ascontiguousarray(rho, dtype=np.float64)
    c = None if chi is None else np.ascontiguousarray(chi, dtype=np.float64)
    phi = np.zeros(n_cells + 1, dtype=np.float64)
    lib().orc_solve_periodic(int(n_cells), float(dx), _ptr(r, ctypes.c_double),
                             _ptr(c, ctypes.c_double), _ptr(phi, ctypes.c_double))
    return phi


def fields(cfg, phi):
    """(cell-centred E [N], node E [N+1]) from the node potential."""
    p = params(cfg)
    ph = np.ascontiguousarray(phi, dtype=np.float64)
    e_cc = np.zeros(p.n_cells + 1)
    e_node = np.zeros(p.n_cells + 1)
    lib().orc_fields(ctypes.byref(p), _ptr(ph, ctypes.c_double), _ptr(e_cc, ctypes.c_double),
                     _ptr(e_node, ctypes.c_double))
    return e_cc[:p.n_cells], e_node


def gather_ec(cfg, e_cc, xi) -> float:
    p = params(cfg)
    e = np.ascontiguousarray(e_cc, dtype=np.float64)
    return lib().orc_gather_ec(ctypes.byref(p), _ptr(e, ctypes.c_double), float(xi))


def gather_ec3(cfg, e_cc, xi) -> float:
    p = params(cfg)
    e = np.ascontiguousarray(e_cc, dtype=np.float64)
    return lib().orc_gather_ec3(ctypes.byref(p), _ptr(e, ctypes.c_double), float(xi))


def gather_mc(cfg, e_node, xi) -> float:
    p = params(cfg)
    e = np.ascontiguousarray(e_node, dtype=np.float64)
    return lib().orc_gather_mc(ctypes.byref(p), _ptr(e, ctypes.c_double), float(xi))


def grid_nodes(h) -> np.ndarray:
    """Node positions of a non-uniform grid from its cell widths."""
    h = np.ascontiguousarray(h, np.float64)
    x = np.zeros(h.size + 1)
    lib().orc_grid_nodes(h.size, _ptr(h, ctypes.c_double), _ptr(x, ctypes.c_double))
    return x


def locate(h, x_nodes, x):
    """(where, cell, off) of a physical position: where -1 / 0 / 1 below, inside, beyond."""
    h = np.ascontiguousarray(h, np.float64)
    xn = np.ascontiguousarray(x_nodes, np.float64)
    c, o = ctypes.c_int64(), ctypes.c_double()
    w = lib().orc_locate(h.size, _ptr(xn, ctypes.c_double), _ptr(h, ctypes.c_double), float(x),
                         ctypes.byref(c), ctypes.byref(o))
    return int(w), int(c.value), float(o.value)


def solve_dirichlet_h(h, q_node, v_left, chi=None) -> np.ndarray:
    h = np.ascontiguousarray(h, np.float64)
    q = np.ascontiguousarray(q_node, np.float64)
    ch = None if chi is None else np.ascontiguousarray(chi, np.float64)
    phi = np.zeros(h.size + 1)
    lib().orc_solve_dirichlet_h(h.size, _ptr(h, ctypes.c_double), _ptr(q, ctypes.c_double),
                                _ptr(ch, ctypes.c_double), float(v_left), _ptr(phi, ctypes.c_double))
    return phi


def solve_periodic_h(h, q_node, chi=None) -> np.ndarray:
    h = np.ascontiguousarray(h, np.float64)
    q = np.ascontiguousarray(q_node, np.float64)
    ch = None if chi is None else np.ascontiguousarray(chi, np.float64)
    phi = np.zeros(h.size + 1)
    lib().orc_solve_periodic_h(h.size, _ptr(h, ctypes.c_double), _ptr(q, ctypes.c_double),
                               _ptr(ch, ctypes.c_double), _ptr(phi, ctypes.c_double))
    return phi


def gather_ec_h(cfg, u_cc, xi) -> float:
    """Field [V/m] at cell coordinate xi on the non-uniform grid of cfg from
    the cells' voltage drops."""
    p = params(cfg)
    u = np.ascontiguousarray(u_cc, np.float64)
    return float(lib().orc_gather_ec_h(ctypes.byref(p), _ptr(u, ctypes.c_double), float(xi)))


def gather_ec3_h(cfg, u_cc, xi) -> float:
    """m = 3: field [V/m] at cell coordinate xi on the non-uniform grid of
    cfg from the cells' voltage drops."""
    p = params(cfg)
    u = np.ascontiguousarray(u_cc, np.float64)
    return float(lib().orc_gather_ec3_h(ctypes.byref(p), _ptr(u, ctypes.c_double), float(xi)))


def rotate(d, cos_chi, phi) -> np.ndarray:
    dd = np.ascontiguousarray(d, dtype=np.float64)
    out = np.zeros(3)
    lib().orc_rotate(_ptr(dd, ctypes.c_double), float(cos_chi), float(phi),
                     _ptr(out, ctypes.c_double))
    return out


class Sim:
    """Whole-simulation oracle: one FP64 run of the method, step by step."""

    def __init__(self, cfg: dict, cap_e: int | None = None, cap_i: int | None = None):
        self.cfg = dict(cfg)
        self.p = params(cfg)
        npi = int(cfg["np_init"])
        cap_e = cap_e if cap_e is not None else max(1024, int(npi * cfg.get("cap_factor", 2.0)))
        cap_i = cap_i if cap_i is not None else cap_e
        if cfg.get("cell_width") is not None and (
                cfg.get("scheme", "ec_explicit") not in ("ec_explicit", "ec_implicit", "ec3_explicit")
                or not cfg.get("ions_mobile", True)):
            raise ValueError("the non-uniform grid takes the EC schemes and mobile ions")
        self._h = lib().orc_sim_create(ctypes.byref(self.p), int(cap_e), int(cap_i))
        if not self._h:
            raise MemoryError("oracle allocation failed")
        self.n_cells = self.p.n_cells
        self.d = derive(self.p)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().orc_sim_free(h)
            self._h = None

    def load(self, n_e: int, n_i: int):
        if lib().orc_sim_load(self._h, int(n_e), int(n_i)):
            raise ValueError("oracle load exceeds capacity")
        return self

    def set_species(self, species, xi, vx, vy, vz, ids, abar=None, next_id=None, wait=None):
        """Inject a state; `wait` (as get_species returns it) keeps each
        particle's steps to its next null-collision selection, None draws
        them as for particles entering the run at the current step."""
        k = SPECIES.get(species, species)
        xi = np.ascontiguousarray(xi, dtype=np.float64)
        n = len(xi)
        vx = np.ascontiguousarray(vx, dtype=np.float64)
        vy = np.ascontiguousarray(vy, dtype=np.float64)
        vz = np.ascontiguousarray(vz, dtype=np.float64)
        ids = np.ascontiguousarray(ids, dtype=np.uint32)
        ab = None if abar is None else np.ascontiguousarray(abar, dtype=np.float64)
        if next_id is None:
            next_id = int(ids.max()) + 1 if n else 0
        wt = None if wait is None else np.ascontiguousarray(wait, dtype=np.uint32)
        r = lib().orc_sim_set(self._h, k, n, _ptr(xi, ctypes.c_double), _ptr(vx, ctypes.c_double),
                              _ptr(vy, ctypes.c_double), _ptr(vz, ctypes.c_double),
                              _ptr(ids, ctypes.c_uint32), _ptr(ab, ctypes.c_double),
                              int(next_id), _ptr(wt, ctypes.c_uint32))
        if r:
            raise ValueError("oracle set exceeds capacity")
        return self

    def init_field(self, set_abar: bool = True):
        lib().orc_sim_init_field(self._h, int(set_abar))
        return self

    def set_step(self, step: int):
        lib().orc_sim_set_step(self._h, int(step))
        return self

    def step(self, n: int = 1):
        if lib().orc_sim_step(self._h, int(n)):
            raise RuntimeError("oracle step failed (capacity exceeded)")
        return self

    def count(self, species) -> int:
        return int(lib().orc_sim_count(self._h, SPECIES.get(species, species)))

    def get_species(self, species) -> dict:
        k = SPECIES.get(species, species)
        n = self.count(k)
        out = {name: np.zeros(n) for name in ("xi", "vx", "vy", "vz", "abar")}
        out["id"] = np.zeros(n, dtype=np.uint32)
        out["wait"] = np.zeros(n, dtype=np.uint32)
        lib().orc_sim_get(self._h, k, _ptr(out["xi"], ctypes.c_double),
                          _ptr(out["vx"], ctypes.c_double), _ptr(out["vy"], ctypes.c_double),
                          _ptr(out["vz"], ctypes.c_double), _ptr(out["id"], ctypes.c_uint32),
                          _ptr(out["abar"], ctypes.c_double), _ptr(out["wait"], ctypes.c_uint32))
        return out

    def diag(self) -> dict:
        d = Diag()
        lib().orc_sim_diag(self._h, ctypes.byref(d))
        return {
            "count": list(d.count), "wall_count": [list(r) for r in d.wall_count],
            "wall_energy_ev": [list(r) for r in d.wall_energy_ev],
            "coll": list(d.coll), "overflow": list(d.overflow), "births": d.births,
            "ke_x": list(d.ke_x), "ke_perp": list(d.ke_perp),
            "field_energy": d.field_energy,
            "field_energy_push": d.field_energy_push, "power": list(d.power), "step": d.step,
            "n_avg": d.n_avg, "n_diag": d.n_diag,
        }

    def grids(self) -> dict:
        n = self.n_cells
        out = {"rho_q_e": np.zeros(n + 1, dtype=np.int64), "rho_q_i": np.zeros(n + 1, dtype=np.int64),
               "phi": np.zeros(n + 1), "e_cc": np.zeros(n), "chi": np.zeros(n)}
        lib().orc_sim_grids(self._h, _ptr(out["rho_q_e"], ctypes.c_int64),
                            _ptr(out["rho_q_i"], ctypes.c_int64), _ptr(out["phi"], ctypes.c_double),
                            _ptr(out["e_cc"], ctypes.c_double), _ptr(out["chi"], ctypes.c_double))
        return out

    def averages(self) -> dict:
        n = self.n_cells
        out = {"ne": np.zeros(n + 1), "ni": np.zeros(n + 1), "phi": np.zeros(n + 1),
               "heat_e": np.zeros(n), "heat_i": np.zeros(n),
               "eedf": np.zeros(self.p.eedf_bins + 1, dtype=np.int64)}
        lib().orc_sim_averages(self._h, _ptr(out["ne"], ctypes.c_double),
                               _ptr(out["ni"], ctypes.c_double), _ptr(out["phi"], ctypes.c_double),
                               _ptr(out["heat_e"], ctypes.c_double),
                               _ptr(out["heat_i"], ctypes.c_double),
                               _ptr(out["eedf"], ctypes.c_int64))
        return out

    def reset_averages(self):
        lib().orc_sim_reset_averages(self._h)
        return self

    def energy(self) -> float:
        """Total energy [J/m^2] at the time level of the last push: time-centred
        kinetic energy plus the energy of the field that push used."""
        d = self.diag()
        return sum(d["ke_x"]) + sum(d["ke_perp"]) + d["field_energy_push"]


# ---- collisionless EC run and its discrete adjoint (adjoint.c) ----

class AdjProblem(ctypes.Structure):
    _fields_ = [
        ("n_cells", ctypes.c_int32), ("periodic", ctypes.c_int32),
        ("nsteps", ctypes.c_int64), ("step0", ctypes.c_int64),
        ("length", ctypes.c_double), ("dt", ctypes.c_double),
        ("rf_freq", ctypes.c_double), ("rf_volt", ctypes.c_double),
        ("weight", ctypes.c_double), ("bg_density", ctypes.c_double),
        ("c_power", ctypes.c_double), ("c_flux", ctypes.c_double),
    ]


def adj_problem(n_cells, periodic, nsteps, length, dt, rf_freq=0.0, rf_volt=0.0, weight=1.0,
                bg_density=0.0, step0=0, c_power=1.0, c_flux=0.0) -> AdjProblem:
    return AdjProblem(int(n_cells), int(bool(periodic)), int(nsteps), int(step0), float(length),
                      float(dt), float(rf_freq), float(rf_volt), float(weight), float(bg_density),
                      float(c_power), float(c_flux))


def adj_forward(pb: AdjProblem, xi0, vx0) -> dict:
    """Collisionless EC run: time-averaged absorbed power and current density,
    final state and absorption steps (-1: never absorbed)."""
    xi0 = np.ascontiguousarray(xi0, np.float64)
    vx0 = np.ascontiguousarray(vx0, np.float64)
    n = xi0.size
    pw, fl = ctypes.c_double(), ctypes.c_double()
    xe, ve = np.zeros(n), np.zeros(n)
    ab = np.zeros(n, np.int64)
    rc = lib().orc_adj_forward(ctypes.byref(pb), n, _ptr(xi0, ctypes.c_double), _ptr(vx0, ctypes.c_double),
                               ctypes.cast(ctypes.byref(pw), _d), ctypes.cast(ctypes.byref(fl), _d),
                               _ptr(xe, ctypes.c_double), _ptr(ve, ctypes.c_double), _ptr(ab, ctypes.c_int64))
    if rc:
        raise RuntimeError("orc_adj_forward failed")
    return {"power": pw.value, "flux": fl.value, "xi": xe, "vx": ve, "absorbed_at": ab}


def adj_gradient(pb: AdjProblem, xi0, vx0) -> dict:
    """J = c_power <P> + c_flux <Gamma> and dJ/dv^{-1/2}, dJ/dxi^0, dJ/dV0."""
    xi0 = np.ascontiguousarray(xi0, np.float64)
    vx0 = np.ascontiguousarray(vx0, np.float64)
    n = xi0.size
    j, dv0 = ctypes.c_double(), ctypes.c_double()
    gv, gx = np.zeros(n), np.zeros(n)
    rc = lib().orc_adj_gradient(ctypes.byref(pb), n, _ptr(xi0, ctypes.c_double), _ptr(vx0, ctypes.c_double),
                                ctypes.cast(ctypes.byref(j), _d), _ptr(gv, ctypes.c_double),
                                _ptr(gx, ctypes.c_double), ctypes.cast(ctypes.byref(dv0), _d))
    if rc:
        raise RuntimeError("orc_adj_gradient failed")
    return {"J": j.value, "dvx0": gv, "dxi0": gx, "dV0": dv0.value}
