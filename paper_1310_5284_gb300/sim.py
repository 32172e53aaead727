"""Python binding of one run: builds the pic_config from a workload dict, owns
the device arena as a torch tensor, and forwards every call to libpic.so.

PyTorch only supplies device memory and the CUDA stream; all arithmetic of
the method runs in the library's kernels.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _abi

SPECIES = {"e": 0, "i": 1, 0: 0, 1: 1}


def make_config(cfg: dict) -> _abi.PicConfig:
    """pic_config from a workload description dict (see workloads/__init__.py)."""
    c = _abi.PicConfig()
    c.scheme = _abi.SCHEMES[cfg.get("scheme", "ec_explicit")]
    c.boundary = _abi.BOUNDARY_PERIODIC if cfg.get("periodic", False) else _abi.BOUNDARY_ELECTRODES
    c.n_cells = int(cfg["n_cells"])
    c.mcc = int(bool(cfg.get("mcc", True)))
    c.ions_mobile = int(bool(cfg.get("ions_mobile", True)))
    c.strict = int(bool(cfg.get("strict", False)))
    c.sort_period = int(cfg.get("sort_period", 16))
    c.diag_period = int(cfg.get("diag_period", 0))
    c.eedf_bins = int(cfg.get("eedf_bins", 100))
    c.seed = int(cfg.get("seed", 1)) & 0xffffffff
    c.run = int(cfg.get("run", 0)) & 0xffffffff
    np_init = int(cfg["np_init"])
    c.np_init = np_init
    cap_factor = float(cfg.get("cap_factor", 2.0))
    cap = int(cfg.get("capacity", max(1024, int(np_init * cap_factor))))
    c.capacity[0] = cap
    c.capacity[1] = int(cfg.get("capacity_i", cap)) if c.ions_mobile else 1
    # one step may record the births of up to an eighth of the slots
    c.births_capacity = int(cfg.get("births_capacity", min(1 << 24, max(4096, cap // 8))))
    c.length = float(cfg["length"])
    c.dt = float(cfg["dt"])
    c.rf_freq = float(cfg.get("rf_freq", 0.0))
    c.rf_volt = float(cfg.get("rf_volt", 0.0))
    c.n0 = float(cfg["n0"])
    c.bg_density = float(cfg.get("bg_density", 0.0))
    c.te_ev = float(cfg.get("te_ev", 2.0))
    c.ti_ev = float(cfg.get("ti_ev", 0.026))
    c.ion_mass_amu = float(cfg.get("ion_mass_amu", 39.948))
    c.pressure_mtorr = float(cfg.get("pressure_mtorr", 0.0))
    c.gas_temp = float(cfg.get("gas_temp", 300.0))
    c.sig_el = float(cfg.get("sig_el", 1e-19))
    c.exc_thr = float(cfg.get("exc_thr", 11.5))
    c.exc_ramp_end = float(cfg.get("exc_ramp_end", 23.0))
    c.sig_exc_max = float(cfg.get("sig_exc_max", 5e-21))
    c.iz_thr = float(cfg.get("iz_thr", 15.8))
    c.sig_iz_peak = float(cfg.get("sig_iz_peak", 3e-20))
    c.sig_cx = float(cfg.get("sig_cx", 5e-19))
    c.eps_cap = float(cfg.get("eps_cap", 100.0))
    c.cx_vmax = float(cfg.get("cx_vmax", 2.0 * c.rf_volt + 50.0))
    c.eedf_max_ev = float(cfg.get("eedf_max_ev", 50.0))
    c.collision_model = (_abi.IZ_OPAL if cfg.get("iz_split", "equal") == "opal" else 0) | \
        (_abi.SCATTER_VS if cfg.get("scattering", "isotropic") == "vahedi_surendra" else 0)
    c.iz_split_b = float(cfg.get("iz_split_b", 10.0))
    if cfg.get("cell_width") is not None:
        # non-uniform grid: the array stays referenced by the struct
        import numpy as np

        h = np.ascontiguousarray(cfg["cell_width"], dtype=np.float64)
        if h.shape != (c.n_cells,):
            raise ValueError("cell_width must hold n_cells widths")
        c._cell_width = h
        c.cell_width = h.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    return c


def required_sizes(cfg: dict) -> tuple[int, int]:
    c = make_config(cfg)
    s = _abi.PicSizes()
    _abi.check(_abi.lib().pic_required_sizes(ctypes.byref(c), ctypes.byref(s)))
    return int(s.arena_bytes), int(s.snapshot_bytes)


def _fptr(a, ct):
    return None if a is None else a.ctypes.data_as(ctypes.POINTER(ct))


class Sim:
    """One discharge run on one GPU (pic_init / pic_step / pic_diag)."""

    def __init__(self, cfg: dict, device="cuda", stream=None):
        import torch

        self.cfg = dict(cfg)
        self._c = make_config(cfg)
        self.n_cells = self._c.n_cells
        self.device = torch.device(device)
        arena_bytes, self.snapshot_bytes = required_sizes(cfg)
        with torch.cuda.device(self.device):
            self.arena = torch.empty(arena_bytes, dtype=torch.uint8, device=self.device)
            self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        bufs = _abi.PicBuffers(self.arena.data_ptr(), arena_bytes)
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            _abi.check(_abi.lib().pic_init(ctypes.byref(self._c), ctypes.byref(bufs),
                                           ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h)))
        self._h = h

    # ---- lifecycle ----
    def close(self):
        h = getattr(self, "_h", None)
        if h:
            _abi.lib().pic_free(h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, code):
        return _abi.check(code, self._h)

    # ---- stepping ----
    def step(self, n: int = 1):
        self._check(_abi.lib().pic_step(self._h, int(n)))
        return self

    def init_field(self, set_abar: bool = True):
        self._check(_abi.lib().pic_init_field(self._h, int(bool(set_abar))))
        return self

    def set_step(self, step: int):
        self._check(_abi.lib().pic_set_step(self._h, int(step)))
        return self

    # ---- diagnostics ----
    def diag(self, reset_avg: bool = False) -> dict:
        d = _abi.PicDiag()
        self._check(_abi.lib().pic_diag(self._h, ctypes.byref(d), int(bool(reset_avg))))
        return {
            "step": d.step, "count": list(d.count),
            "wall_count": [list(r) for r in d.wall_count],
            "wall_energy_ev": [list(r) for r in d.wall_energy_ev],
            "coll": list(d.coll), "overflow": list(d.overflow), "births": d.births,
            "ke_x": list(d.ke_x), "ke_perp": list(d.ke_perp), "field_energy": d.field_energy,
            "field_energy_push": d.field_energy_push, "power": list(d.power),
            "n_avg": d.n_avg, "n_diag": d.n_diag, "status": d.status,
        }

    def energy(self) -> float:
        d = self.diag()
        return sum(d["ke_x"]) + sum(d["ke_perp"]) + d["field_energy_push"]

    def profiles(self) -> dict:
        n = self.n_cells
        out = {k: np.zeros(n + 1) for k in ("ne", "ni", "phi")}
        out["heat_e"] = np.zeros(n)
        out["heat_i"] = np.zeros(n)
        out["eedf"] = np.zeros(self._c.eedf_bins + 1, dtype=np.uint64)
        self._check(_abi.lib().pic_profiles(
            self._h, out["ne"].ctypes.data, out["ni"].ctypes.data, out["phi"].ctypes.data,
            out["heat_e"].ctypes.data, out["heat_i"].ctypes.data, out["eedf"].ctypes.data))
        return out

    def grids(self) -> dict:
        n = self.n_cells
        out = {"rho_q_e": np.zeros(n + 1, dtype=np.int64), "rho_q_i": np.zeros(n + 1, dtype=np.int64),
               "phi": np.zeros(n + 1), "e_cc": np.zeros(n), "chi": np.zeros(n)}
        self._check(_abi.lib().pic_grids(self._h, out["rho_q_e"].ctypes.data,
                                         out["rho_q_i"].ctypes.data, out["phi"].ctypes.data,
                                         out["e_cc"].ctypes.data, out["chi"].ctypes.data))
        return out

    def count(self) -> tuple[int, int]:
        a, b = ctypes.c_int64(), ctypes.c_int64()
        self._check(_abi.lib().pic_count(self._h, ctypes.byref(a), ctypes.byref(b)))
        return a.value, b.value

    def status(self) -> int:
        s = ctypes.c_uint32()
        self._check(_abi.lib().pic_status(self._h, ctypes.byref(s)))
        return s.value

    # ---- particles ----
    def get_particles(self, species) -> dict:
        k = SPECIES[species]
        n = self.count()[k]
        out = {"cell": np.zeros(n, np.int32), "off": np.zeros(n, np.float32),
               "vx": np.zeros(n, np.float32), "vy": np.zeros(n, np.float32),
               "vz": np.zeros(n, np.float32), "id": np.zeros(n, np.uint32),
               "abar": np.zeros(n, np.float32)}
        hp = _abi.PicHostParticles(n, _fptr(out["cell"], ctypes.c_int32), _fptr(out["off"], ctypes.c_float),
                                   _fptr(out["vx"], ctypes.c_float), _fptr(out["vy"], ctypes.c_float),
                                   _fptr(out["vz"], ctypes.c_float), _fptr(out["id"], ctypes.c_uint32),
                                   _fptr(out["abar"], ctypes.c_float), 0)
        self._check(_abi.lib().pic_get_particles(self._h, k, ctypes.byref(hp)))
        m = int(hp.count)
        res = {name: arr[:m] for name, arr in out.items()}
        res["next_id"] = int(hp.next_id)
        return res

    @staticmethod
    def _host_particles(state: dict, next_id: int | None):
        """(pic_host_particles, the arrays it points into) for one species."""
        arrs = {
            "cell": np.ascontiguousarray(state["cell"], np.int32),
            "off": np.ascontiguousarray(state["off"], np.float32),
            "vx": np.ascontiguousarray(state["vx"], np.float32),
            "vy": np.ascontiguousarray(state["vy"], np.float32),
            "vz": np.ascontiguousarray(state["vz"], np.float32),
            "id": np.ascontiguousarray(state["id"], np.uint32),
        }
        ab = state.get("abar")
        arrs["abar"] = None if ab is None else np.ascontiguousarray(ab, np.float32)
        n = len(arrs["cell"])
        if next_id is None:
            next_id = int(arrs["id"].max()) + 1 if n else 0
        hp = _abi.PicHostParticles(n, _fptr(arrs["cell"], ctypes.c_int32), _fptr(arrs["off"], ctypes.c_float),
                                   _fptr(arrs["vx"], ctypes.c_float), _fptr(arrs["vy"], ctypes.c_float),
                                   _fptr(arrs["vz"], ctypes.c_float), _fptr(arrs["id"], ctypes.c_uint32),
                                   _fptr(arrs["abar"], ctypes.c_float), int(next_id))
        return hp, arrs

    def set_particles(self, species, state: dict, next_id: int | None = None):
        hp, _arrs = self._host_particles(state, next_id)
        self._check(_abi.lib().pic_set_particles(self._h, SPECIES[species], ctypes.byref(hp)))
        return self

    def set_state(self, electrons: dict, ions: dict, next_id_e: int | None = None, next_id_i: int | None = None):
        """Both species in one call (pic_set_state): neither changes if a
        particle of either is off the grid."""
        he, _ae = self._host_particles(electrons, next_id_e)
        hi, _ai = self._host_particles(ions, next_id_i)
        self._check(_abi.lib().pic_set_state(self._h, ctypes.byref(he), ctypes.byref(hi)))
        return self

    # ---- checkpoint ----
    def save(self) -> np.ndarray:
        buf = np.empty(self.snapshot_bytes, dtype=np.uint8)
        self._check(_abi.lib().pic_save(self._h, buf.ctypes.data, buf.nbytes))
        return buf

    def load(self, buf: np.ndarray):
        buf = np.ascontiguousarray(buf, dtype=np.uint8)
        self._check(_abi.lib().pic_load(self._h, buf.ctypes.data, buf.nbytes))
        return self


def philox_fill(key, ctr0, n, out_tensor, stream=None):
    """Fill a CUDA uint32/int32 tensor of 4n words with Philox4x32-10 blocks."""
    import torch

    s = stream if stream is not None else torch.cuda.current_stream()
    _abi.check(_abi.lib().pic_philox_fill(int(key[0]), int(key[1]), int(ctr0[0]), int(ctr0[1]),
                                          int(ctr0[2]), int(ctr0[3]), int(n), out_tensor.data_ptr(),
                                          ctypes.c_void_p(s.cuda_stream)))
