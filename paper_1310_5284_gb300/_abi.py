"""ctypes mirror of include/pic.h and the loader of the in-tree libpic.so.

Argument marshalling only: every step of the method runs in the library's
CUDA kernels.  Importing this module on a machine where the library was not
built raises; there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
# PIC_LIBRARY selects an alternative build of the same sources (launch-shape sweeps)
LIB_PATH = os.environ.get("PIC_LIBRARY") or os.path.join(_PKG, "libpic.so")

PIC_OK = 0
ERRORS = {-1: "PIC_EINVAL", -2: "PIC_EUNSTABLE", -3: "PIC_ENOMEM", -4: "PIC_EOVERFLOW",
          -5: "PIC_ECUDA", -6: "PIC_ETIMEOUT"}
PIC_STATUS_CAPACITY, PIC_STATUS_BIRTHS, PIC_STATUS_TIMEOUT = 0x1, 0x2, 0x4
SCHEMES = {"ec_explicit": 0, "mc_explicit": 1, "ec_implicit": 2, "mc_implicit": 3, "ec3_explicit": 4}
BOUNDARY_ELECTRODES, BOUNDARY_PERIODIC = 0, 1
IZ_OPAL, SCATTER_VS = 1, 2  # collision-model option bits


class PicConfig(ctypes.Structure):
    _fields_ = [
        ("scheme", ctypes.c_int32), ("boundary", ctypes.c_int32), ("n_cells", ctypes.c_int32),
        ("mcc", ctypes.c_int32), ("ions_mobile", ctypes.c_int32), ("strict", ctypes.c_int32),
        ("sort_period", ctypes.c_int32), ("diag_period", ctypes.c_int32),
        ("eedf_bins", ctypes.c_int32), ("seed", ctypes.c_uint32), ("run", ctypes.c_uint32),
        ("collision_model", ctypes.c_int32), ("np_init", ctypes.c_int64),
        ("capacity", ctypes.c_int64 * 2), ("births_capacity", ctypes.c_int64),
        ("length", ctypes.c_double), ("dt", ctypes.c_double), ("rf_freq", ctypes.c_double),
        ("rf_volt", ctypes.c_double), ("n0", ctypes.c_double), ("bg_density", ctypes.c_double),
        ("te_ev", ctypes.c_double), ("ti_ev", ctypes.c_double), ("ion_mass_amu", ctypes.c_double),
        ("pressure_mtorr", ctypes.c_double), ("gas_temp", ctypes.c_double),
        ("sig_el", ctypes.c_double), ("exc_thr", ctypes.c_double), ("exc_ramp_end", ctypes.c_double),
        ("sig_exc_max", ctypes.c_double), ("iz_thr", ctypes.c_double),
        ("sig_iz_peak", ctypes.c_double), ("sig_cx", ctypes.c_double), ("eps_cap", ctypes.c_double),
        ("cx_vmax", ctypes.c_double), ("eedf_max_ev", ctypes.c_double), ("iz_split_b", ctypes.c_double),
        ("cell_width", ctypes.POINTER(ctypes.c_double)),
    ]


class PicSizes(ctypes.Structure):
    _fields_ = [("arena_bytes", ctypes.c_size_t), ("snapshot_bytes", ctypes.c_size_t)]


class PicBuffers(ctypes.Structure):
    _fields_ = [("arena", ctypes.c_void_p), ("arena_bytes", ctypes.c_size_t)]


class PicHostParticles(ctypes.Structure):
    _fields_ = [
        ("count", ctypes.c_int64), ("cell", ctypes.POINTER(ctypes.c_int32)),
        ("off", ctypes.POINTER(ctypes.c_float)), ("vx", ctypes.POINTER(ctypes.c_float)),
        ("vy", ctypes.POINTER(ctypes.c_float)), ("vz", ctypes.POINTER(ctypes.c_float)),
        ("id", ctypes.POINTER(ctypes.c_uint32)), ("abar", ctypes.POINTER(ctypes.c_float)),
        ("next_id", ctypes.c_uint32),
    ]


class PicDiag(ctypes.Structure):
    _fields_ = [
        ("step", ctypes.c_int64), ("count", ctypes.c_int64 * 2),
        ("wall_count", (ctypes.c_uint64 * 2) * 2), ("wall_energy_ev", (ctypes.c_double * 2) * 2),
        ("coll", ctypes.c_uint64 * 5), ("overflow", ctypes.c_uint64 * 2), ("births", ctypes.c_uint64),
        ("ke_x", ctypes.c_double * 2), ("ke_perp", ctypes.c_double * 2),
        ("field_energy", ctypes.c_double), ("field_energy_push", ctypes.c_double),
        ("power", ctypes.c_double * 2), ("n_avg", ctypes.c_int64), ("n_diag", ctypes.c_int64),
        ("status", ctypes.c_uint32), ("reserved", ctypes.c_uint32),
    ]


# exported names and signatures, in the order include/pic.h declares them
_P = ctypes.POINTER
_vp = ctypes.c_void_p
class PicAdjConfig(ctypes.Structure):
    _fields_ = [
        ("boundary", ctypes.c_int32), ("n_cells", ctypes.c_int32),
        ("checkpoint_every", ctypes.c_int32), ("reserved0", ctypes.c_int32),
        ("n_particles", ctypes.c_int64), ("nsteps", ctypes.c_int64), ("step0", ctypes.c_int64),
        ("length", ctypes.c_double), ("dt", ctypes.c_double), ("rf_freq", ctypes.c_double),
        ("n0", ctypes.c_double), ("bg_density", ctypes.c_double),
    ]


SIGNATURES = {
    "pic_version": ([], ctypes.c_int),
    "pic_build_info": ([], ctypes.c_char_p),
    "pic_required_sizes": ([_P(PicConfig), _P(PicSizes)], ctypes.c_int),
    "pic_init": ([_P(PicConfig), _P(PicBuffers), _vp, _P(_vp)], ctypes.c_int),
    "pic_step": ([_vp, ctypes.c_int64], ctypes.c_int),
    "pic_diag": ([_vp, _P(PicDiag), ctypes.c_int], ctypes.c_int),
    "pic_profiles": ([_vp, _vp, _vp, _vp, _vp, _vp, _vp], ctypes.c_int),
    "pic_grids": ([_vp, _vp, _vp, _vp, _vp, _vp], ctypes.c_int),
    "pic_count": ([_vp, _P(ctypes.c_int64), _P(ctypes.c_int64)], ctypes.c_int),
    "pic_get_particles": ([_vp, ctypes.c_int, _P(PicHostParticles)], ctypes.c_int),
    "pic_set_particles": ([_vp, ctypes.c_int, _P(PicHostParticles)], ctypes.c_int),
    "pic_set_state": ([_vp, _P(PicHostParticles), _P(PicHostParticles)], ctypes.c_int),
    "pic_selftest_wait": ([ctypes.c_int64, _P(ctypes.c_uint32), _P(ctypes.c_double), _vp], ctypes.c_int),
    "pic_init_field": ([_vp, ctypes.c_int], ctypes.c_int),
    "pic_set_step": ([_vp, ctypes.c_int64], ctypes.c_int),
    "pic_status": ([_vp, _P(ctypes.c_uint32)], ctypes.c_int),
    "pic_save": ([_vp, _vp, ctypes.c_size_t], ctypes.c_int),
    "pic_load": ([_vp, _vp, ctypes.c_size_t], ctypes.c_int),
    "pic_philox_fill": ([ctypes.c_uint32] * 6 + [ctypes.c_int64, _vp, _vp], ctypes.c_int),
    "pic_batch_required_sizes": ([_vp, ctypes.c_int32, _P(PicSizes)], ctypes.c_int),
    "pic_batch_init": ([_vp, ctypes.c_int32, _P(PicBuffers), _vp, _P(_vp)], ctypes.c_int),
    "pic_batch_step": ([_vp, ctypes.c_int64], ctypes.c_int),
    "pic_batch_diag": ([_vp, ctypes.c_int32, _P(PicDiag), ctypes.c_int], ctypes.c_int),
    "pic_batch_get_particles": ([_vp, ctypes.c_int32, ctypes.c_int, _P(PicHostParticles)], ctypes.c_int),
    "pic_batch_profiles": ([_vp, ctypes.c_int32, _vp, _vp, _vp, _vp, _vp, _vp], ctypes.c_int),
    "pic_batch_set_schedule": ([_vp, ctypes.c_int64, ctypes.c_int32], ctypes.c_int),
    "pic_batch_autotune": ([_vp, ctypes.c_int32, _P(ctypes.c_int64), _P(ctypes.c_int32),
                            _P(ctypes.c_double)], ctypes.c_int),
    "pic_batch_status": ([_vp, _P(ctypes.c_uint32)], ctypes.c_int),
    "pic_batch_free": ([_vp], None),
    "pic_adj_required_sizes": ([_P(PicAdjConfig), _P(PicSizes)], ctypes.c_int),
    "pic_adj_init": ([_P(PicAdjConfig), _P(PicBuffers), _vp, _P(_vp)], ctypes.c_int),
    "pic_adj_forward": ([_vp, ctypes.c_double, _vp, _vp, _vp, _P(ctypes.c_double)], ctypes.c_int),
    "pic_adj_backward": ([_vp, ctypes.c_double, ctypes.c_double, _vp, _vp, _P(ctypes.c_double)], ctypes.c_int),
    "pic_adj_final_state": ([_vp, _vp, _vp, _vp], ctypes.c_int),
    "pic_adj_free": ([_vp], None),
    "pic_deposit_noalloc": ([ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _vp, _vp, ctypes.c_int64,
                             _vp, _vp], ctypes.c_int),
    "pic_free": ([_vp], None),
    "pic_last_error": ([_vp], ctypes.c_char_p),
}

_lib = None


def lib():
    """The loaded library.  Raises if libpic.so has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("libpic.so not built (run __graft_entry__.build() or "
                              "python -m paper_1310_5284_gb300.build): %s" % LIB_PATH)
        L = ctypes.CDLL(LIB_PATH)
        for name, (args, res) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res
        _lib = L
    return _lib


class PicError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s: %s" % (ERRORS.get(code, code), msg))
        self.code = code


def check(code, handle=None):
    if code != PIC_OK:
        msg = lib().pic_last_error(handle)
        raise PicError(code, msg.decode() if msg else "")
    return code
