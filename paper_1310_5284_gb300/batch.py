"""Python binding of a batch of independent runs (pic_batch_* in include/pic.h).

Argument marshalling only; the runs advance in the library's persistent
batched kernels.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _abi
from .sim import SPECIES, _fptr, make_config

class BatchSim:
    """Many runs advanced together (pic_batch_init / pic_batch_step)."""

    def __init__(self, cfgs: list[dict], device="cuda", stream=None):
        import torch

        self.cfgs = [dict(c) for c in cfgs]
        arr = (_abi.PicConfig * len(cfgs))(*[make_config(c) for c in cfgs])
        self._arr = arr
        sizes = _abi.PicSizes()
        _abi.check(_abi.lib().pic_batch_required_sizes(arr, len(cfgs), ctypes.byref(sizes)))
        self.device = torch.device(device)
        with torch.cuda.device(self.device):
            self.arena = torch.empty(int(sizes.arena_bytes), dtype=torch.uint8, device=self.device)
            self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        bufs = _abi.PicBuffers(self.arena.data_ptr(), int(sizes.arena_bytes))
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            _abi.check(_abi.lib().pic_batch_init(arr, len(cfgs), ctypes.byref(bufs),
                                                 ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h)))
        self._h = h

    def close(self):
        h = getattr(self, "_h", None)
        if h:
            _abi.lib().pic_batch_free(h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, n: int = 1):
        _abi.check(_abi.lib().pic_batch_step(self._h, int(n)))
        return self

    def set_schedule(self, chunk: int, sort_period: int):
        _abi.check(_abi.lib().pic_batch_set_schedule(self._h, int(chunk), int(sort_period)))
        return self

    def autotune(self, trial_steps: int = 8) -> dict:
        ch, sp, ms = ctypes.c_int64(), ctypes.c_int32(), ctypes.c_double()
        _abi.check(_abi.lib().pic_batch_autotune(self._h, int(trial_steps), ctypes.byref(ch),
                                                 ctypes.byref(sp), ctypes.byref(ms)))
        return {"chunk": ch.value, "sort_period": sp.value, "ms_per_step": ms.value}

    def status(self) -> int:
        s = ctypes.c_uint32()
        _abi.check(_abi.lib().pic_batch_status(self._h, ctypes.byref(s)))
        return s.value

    def diag(self, run: int, reset_avg: bool = False) -> dict:
        d = _abi.PicDiag()
        _abi.check(_abi.lib().pic_batch_diag(self._h, int(run), ctypes.byref(d), int(bool(reset_avg))))
        return {"step": d.step, "count": list(d.count), "coll": list(d.coll), "births": d.births,
                "wall_count": [list(r) for r in d.wall_count], "ke_x": list(d.ke_x),
                "ke_perp": list(d.ke_perp), "field_energy": d.field_energy,
                "field_energy_push": d.field_energy_push, "status": d.status}

    def profiles(self, run: int) -> dict:
        """Time-averaged profiles of one run since its last reset (as Sim.profiles)."""
        c = self.cfgs[run]
        n = int(c["n_cells"])
        out = {k: np.zeros(n + 1) for k in ("ne", "ni", "phi")}
        out["heat_e"] = np.zeros(n)
        out["heat_i"] = np.zeros(n)
        out["eedf"] = np.zeros(int(c.get("eedf_bins", 100)) + 1, dtype=np.uint64)
        _abi.check(_abi.lib().pic_batch_profiles(
            self._h, int(run), out["ne"].ctypes.data, out["ni"].ctypes.data, out["phi"].ctypes.data,
            out["heat_e"].ctypes.data, out["heat_i"].ctypes.data, out["eedf"].ctypes.data))
        return out

    def get_particles(self, run: int, species) -> dict:
        k = SPECIES[species]
        n = self.diag(run)["count"][k]
        out = {"cell": np.zeros(n, np.int32), "off": np.zeros(n, np.float32),
               "vx": np.zeros(n, np.float32), "vy": np.zeros(n, np.float32),
               "vz": np.zeros(n, np.float32), "id": np.zeros(n, np.uint32),
               "abar": np.zeros(n, np.float32)}
        hp = _abi.PicHostParticles(n, _fptr(out["cell"], ctypes.c_int32), _fptr(out["off"], ctypes.c_float),
                                   _fptr(out["vx"], ctypes.c_float), _fptr(out["vy"], ctypes.c_float),
                                   _fptr(out["vz"], ctypes.c_float), _fptr(out["id"], ctypes.c_uint32),
                                   _fptr(out["abar"], ctypes.c_float), 0)
        _abi.check(_abi.lib().pic_batch_get_particles(self._h, int(run), k, ctypes.byref(hp)))
        m = int(hp.count)
        return {name: arr[:m] for name, arr in out.items()}
